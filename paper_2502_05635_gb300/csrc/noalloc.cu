// Low-rank kernel contraction of Eq. svd_acc that allocates nothing:
// y = diag o x + U (S o (V^H x)) on caller-owned device arrays, with its intermediate
// vectors in a fixed, file-scope device array instead of memory from cudaMalloc.
//
// Who needs this: callers that must not allocate device memory on the call path -- code
// whose device memory is owned by another framework's pool (a plain cudaMalloc would
// bypass that pool's accounting and limits), loops that cannot afford the implicit device
// synchronisation of cudaMalloc/cudaFree, and callers that run close to a hard memory cap
// where an allocation could fail mid-run.  They pass every input and output; the only
// other memory used is the array below, reserved once per device when the library loads.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "common.cuh"

namespace tdagw {

namespace {

// Largest supported rank, and the number of row blocks of the V^H x pass.
constexpr int kNoallocMaxRank = 2048;
constexpr int kNoallocBlocks = 152;
// Scratch: kNoallocBlocks partial vectors of length rank, then S o (V^H x) (rank entries):
// (152 + 1) x 2048 complex64 = 2.4 MiB on every device that loads the library.
constexpr size_t kNoallocScratchElems = (size_t)(kNoallocBlocks + 1) * kNoallocMaxRank;

static __device__ __align__(256) float2 g_noalloc_scratch[kNoallocScratchElems];

// Device addresses of the scratch array, looked up once per device (host code may not use
// the symbol itself as a device pointer).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Every array must live on the device the work is launched on (the current one): the
// kernels and the scratch address are per device, so a pointer into another GPU's memory
// or into host memory is rejected instead of being dereferenced across the bus.
void require_on_device(const void* p, int dev, const char* name) {
    cudaPointerAttributes a{};
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        throw Error(TDAGW_ERR_INVALID_ARG, std::string(name) + ": not a CUDA pointer (" +
                                               cudaGetErrorString(e) + ")");
    }
    const bool ok = (a.type == cudaMemoryTypeDevice && a.device == dev) ||
                    a.type == cudaMemoryTypeManaged;
    TDAGW_REQUIRE(ok, TDAGW_ERR_INVALID_ARG,
                  std::string(name) + " is not device memory of the current device (" +
                      std::to_string(dev) + ")");
}

float2* scratch_for_device(int dev) {
    TDAGW_REQUIRE(dev >= 0 && dev < kMaxDevices, TDAGW_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            throw Error(TDAGW_ERR_CUDA,
                        std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    return static_cast<float2*>(g_scratch_ptr[dev]);
}

}  // namespace

}  // namespace tdagw

using namespace tdagw;

extern "C" int tdagw_apply_lowrank_noalloc(const void* U, const void* V, int64_t ld,
                                           const float* S, const void* diag, int64_t N,
                                           int rank, const void* x, void* y, void* stream) {
    try {
        TDAGW_REQUIRE(U && V && S && diag && x && y, TDAGW_ERR_INVALID_ARG, "NULL argument");
        TDAGW_REQUIRE(N >= 1, TDAGW_ERR_INVALID_ARG, "N must be positive");
        TDAGW_REQUIRE(rank >= 1 && rank <= kNoallocMaxRank, TDAGW_ERR_INVALID_ARG,
                      "rank must be in [1, 2048] for the allocation-free apply");
        TDAGW_REQUIRE(ld >= rank && (ld % 2) == 0, TDAGW_ERR_INVALID_ARG,
                      "ld must be even and >= rank");
        TDAGW_REQUIRE(((uintptr_t)U % 16 == 0) && ((uintptr_t)V % 16 == 0) &&
                          ((uintptr_t)x % 16 == 0) && ((uintptr_t)y % 16 == 0),
                      TDAGW_ERR_INVALID_ARG, "U, V, x and y must be 16-byte aligned");
        TDAGW_REQUIRE(x != y, TDAGW_ERR_INVALID_ARG, "x and y must not alias");
        int dev = 0;
        TDAGW_CUDA(cudaGetDevice(&dev));
        const void* arrays[6] = {U, V, S, diag, x, y};
        const char* names[6] = {"U", "V", "S", "diag", "x", "y"};
        for (int i = 0; i < 6; ++i) require_on_device(arrays[i], dev, names[i]);
        float2* scratch = scratch_for_device(dev);
        float2* part = scratch;                                        // blocks x rank
        float2* ytil = scratch + (size_t)kNoallocBlocks * kNoallocMaxRank;  // rank
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        // every partial entry and every used entry of ytil is written before it is read,
        // so nothing in the shared scratch has to be cleared between calls
        const int nblocks = (int)(N < kNoallocBlocks ? N : kNoallocBlocks);
        launch_vcols<float>(V, ld, N, rank, x, part, nblocks, s);
        launch_yreduce<float>(part, nblocks, rank, S, ytil, s);
        launch_gemv<float>(U, ld, N, rank, ytil, y, 1, diag, x, s);
        last_error_message().clear();
        return TDAGW_OK;
    } catch (const Error& e) {
        last_error_message() = e.what();
        return e.code;
    } catch (const std::exception& e) {
        last_error_message() = e.what();
        return TDAGW_ERR_CUDA;
    }
}
