// host_mem.cu -- page-locked host memory for levels held in host memory and
// streamed through the device (the pipeline's host side; the paper keeps
// its out-of-core data in host memory and on disks, Sec. 3).
//
// A level of the 1024^3 configuration is 21.5 GB per copy.  The allocation
// maps it anonymously, asks the kernel for transparent huge pages
// (madvise(MADV_HUGEPAGE): 512 MB pages on a 64 KB-page kernel, 2 MB on a
// 4 KB one), faults every page in with several host threads (zero-filled),
// and registers the range with CUDA, so that device copies from and to it are
// page-locked and asynchronous.  Huge-page backing keeps the number of
// translations the copies walk small whatever the state of the host's free
// memory; the CUDA host allocator's own pinned memory is backed by base pages.
#include <cuda_runtime.h>
#include <sys/mman.h>
#include <unistd.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "abi_common.h"

namespace {

struct Mapping {
    void* base;     // what mmap returned
    size_t length;  // what was mapped
};

std::mutex g_mu;
std::unordered_map<void*, Mapping> g_maps;

size_t huge_page_bytes() {
    size_t v = 0;
    if (FILE* f = std::fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
        unsigned long long x = 0;
        if (std::fscanf(f, "%llu", &x) == 1) v = size_t(x);
        std::fclose(f);
    }
    return (v >= 4096 && (v & (v - 1)) == 0) ? v : size_t(2) << 20;
}

}  // namespace

extern "C" int gamer_host_alloc(size_t bytes, int32_t nthreads, void** out) {
    using namespace gamer;
    if (!out) return GAMER_E_NULL;
    *out = nullptr;
    if (bytes == 0 || bytes > (size_t(1) << 46)) return GAMER_E_PARAM;
    const size_t hp = huge_page_bytes();
    const size_t len = (bytes + hp - 1) / hp * hp;
    // over-map by one huge page so that the range can start on a huge-page
    // boundary
    void* base = mmap(nullptr, len + hp, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS,
                      -1, 0);
    if (base == MAP_FAILED) return GAMER_E_CUDA;
    char* p = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(base) + hp - 1) / hp * hp);
    madvise(p, len, MADV_HUGEPAGE);  // a request: base pages where it cannot be met
    // first touch from several threads
    int nt = nthreads > 0 ? nthreads : int(std::thread::hardware_concurrency());
    nt = std::max(1, std::min(nt, 64));
    const size_t chunk = (len / hp + nt - 1) / nt * hp;
    // (no exception may cross the C ABI: where a thread cannot be started,
    // the calling thread touches that chunk itself)
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t) {
        const size_t lo = size_t(t) * chunk;
        if (lo >= len) break;
        const size_t n = std::min(chunk, len - lo);
        try {
            th.emplace_back([p, lo, n] { std::memset(p + lo, 0, n); });
        } catch (...) {
            std::memset(p + lo, 0, n);
        }
    }
    for (auto& x : th) x.join();
    if (cudaHostRegister(p, len, cudaHostRegisterDefault) != cudaSuccess) {
        cudaGetLastError();
        munmap(base, len + hp);
        return GAMER_E_CUDA;
    }
    try {
        std::lock_guard<std::mutex> lock(g_mu);
        g_maps[p] = Mapping{base, len + hp};
    } catch (...) {
        cudaHostUnregister(p);
        munmap(base, len + hp);
        return GAMER_E_CUDA;
    }
    *out = p;
    return GAMER_OK;
}

extern "C" int gamer_host_free(void* ptr) {
    if (!ptr) return GAMER_E_NULL;
    Mapping m;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_maps.find(ptr);
        if (it == g_maps.end()) return GAMER_E_PARAM;
        m = it->second;
        g_maps.erase(it);
    }
    const bool ok = cudaHostUnregister(ptr) == cudaSuccess;
    if (!ok) cudaGetLastError();
    munmap(m.base, m.length);
    return ok ? GAMER_OK : GAMER_E_CUDA;
}
