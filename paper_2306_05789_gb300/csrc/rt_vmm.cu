// rt_vmm.cu -- growable device buffers on the CUDA virtual memory interface.
//
// The far field of a large operator is assembled wave by wave (a bounded set
// of ACA blocks at a time) and packed as each wave finishes.  Its final size
// is known only at the end, so its storage is a reserved address range that
// receives physical memory as it grows: nothing is copied, and the ACA
// scratch of only one wave is alive at a time.  The driver entry points are
// looked up through the runtime, so the library does not link libcuda.
#include <cuda.h>

#include <mutex>
#include <string>

#include "rt_internal.h"

namespace rt {

namespace {

struct VmmApi {
    CUresult (*reserve)(CUdeviceptr*, size_t, size_t, CUdeviceptr, unsigned long long) = nullptr;
    CUresult (*addr_free)(CUdeviceptr, size_t) = nullptr;
    CUresult (*create)(CUmemGenericAllocationHandle*, size_t, const CUmemAllocationProp*, unsigned long long) = nullptr;
    CUresult (*release)(CUmemGenericAllocationHandle) = nullptr;
    CUresult (*map)(CUdeviceptr, size_t, size_t, CUmemGenericAllocationHandle, unsigned long long) = nullptr;
    CUresult (*unmap)(CUdeviceptr, size_t) = nullptr;
    CUresult (*set_access)(CUdeviceptr, size_t, const CUmemAccessDesc*, size_t) = nullptr;
    CUresult (*granularity)(size_t*, const CUmemAllocationProp*, CUmemAllocationGranularity_flags) = nullptr;
    bool ok = false;
};

template <class F>
bool load_entry(const char* name, F& fn)
{
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
        return false;
    fn = reinterpret_cast<F>(p);
    return true;
}

const VmmApi& api()
{
    static VmmApi a;
    static std::once_flag once;
    std::call_once(once, [] {
        a.ok = load_entry("cuMemAddressReserve", a.reserve) && load_entry("cuMemAddressFree", a.addr_free) &&
               load_entry("cuMemCreate", a.create) && load_entry("cuMemRelease", a.release) &&
               load_entry("cuMemMap", a.map) && load_entry("cuMemUnmap", a.unmap) &&
               load_entry("cuMemSetAccess", a.set_access) &&
               load_entry("cuMemGetAllocationGranularity", a.granularity);
    });
    return a;
}

CUmemAllocationProp device_prop(int device)
{
    CUmemAllocationProp p{};
    p.type = CU_MEM_ALLOCATION_TYPE_PINNED;
    p.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
    p.location.id = device;
    return p;
}

size_t round_up(size_t x, size_t g) { return (x + g - 1) / g * g; }

}  // namespace

int growbuf_reserve(GrowBuf& b, size_t bytes, int device, std::string& err)
{
    const VmmApi& A = api();
    if (!A.ok) {
        err = "virtual memory entry points unavailable";
        return RT_ECUDA;
    }
    const CUmemAllocationProp prop = device_prop(device);
    size_t g = 0;
    if (A.granularity(&g, &prop, CU_MEM_ALLOC_GRANULARITY_RECOMMENDED) != CUDA_SUCCESS || g == 0) {
        err = "cuMemGetAllocationGranularity failed";
        return RT_ECUDA;
    }
    b.gran = g;
    b.device = device;
    b.reserved = round_up(std::max<size_t>(bytes, 1), g);
    CUdeviceptr p = 0;
    if (A.reserve(&p, b.reserved, 0, 0, 0) != CUDA_SUCCESS) {
        err = "cuMemAddressReserve failed";
        b.reserved = 0;
        return RT_ENOMEM;
    }
    b.base = (unsigned long long)p;
    b.mapped = 0;
    return RT_OK;
}

int growbuf_grow(GrowBuf& b, size_t bytes, std::string& err)
{
    const VmmApi& A = api();
    const size_t need = round_up(bytes, b.gran);
    if (need <= b.mapped) return RT_OK;
    if (need > b.reserved) {
        err = "growable buffer: reservation exceeded";
        return RT_EINVAL;
    }
    const size_t chunk = need - b.mapped;
    const CUmemAllocationProp prop = device_prop(b.device);
    CUmemGenericAllocationHandle h = 0;
    if (A.create(&h, chunk, &prop, 0) != CUDA_SUCCESS) {
        err = "cuMemCreate of " + std::to_string(chunk) + " bytes failed";
        return RT_ENOMEM;
    }
    const CUdeviceptr at = (CUdeviceptr)(b.base + b.mapped);
    if (A.map(at, chunk, 0, h, 0) != CUDA_SUCCESS) {
        A.release(h);
        err = "cuMemMap failed";
        return RT_ECUDA;
    }
    CUmemAccessDesc acc{};
    acc.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
    acc.location.id = b.device;
    acc.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
    if (A.set_access(at, chunk, &acc, 1) != CUDA_SUCCESS) {
        A.unmap(at, chunk);
        A.release(h);
        err = "cuMemSetAccess failed";
        return RT_ECUDA;
    }
    b.handles.push_back((unsigned long long)h);
    b.sizes.push_back(chunk);
    b.mapped = need;
    return RT_OK;
}

void growbuf_release(GrowBuf& b)
{
    if (!b.base) return;
    const VmmApi& A = api();
    size_t off = 0;
    for (size_t k = 0; k < b.handles.size(); ++k) {
        A.unmap((CUdeviceptr)(b.base + off), b.sizes[k]);
        A.release((CUmemGenericAllocationHandle)b.handles[k]);
        off += b.sizes[k];
    }
    A.addr_free((CUdeviceptr)b.base, b.reserved);
    b = GrowBuf();
}

}  // namespace rt
