// amg_colour_noalloc: the node colouring of a block-CSR pattern (the one
// amg_setup computes for level 0) without any memory allocation.  For callers
// that may not allocate device memory at the time of the call: code running
// while a stream is being captured into a CUDA graph (cudaMalloc is not
// permitted during capture), allocation-free real-time or callback paths, and
// applications whose device memory is reserved up front by their own
// allocator.  The worklist queues of the colouring kernel live in the
// file-scope device array below instead of memory obtained at run time.
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace bamg {
namespace {

// Scratch: two queues of kWorklistMaxNodes ints, two result ints and the
// pattern-check flag (320,016 bytes).  Every GPU that loads the library holds
// it until the process exits; every call on a device shares it.
constexpr int kNoAllocScratchInts = 2 * kWorklistMaxNodes + 4;
static __device__ __align__(256) int g_colour_scratch[kNoAllocScratchInts];

constexpr int kMaxDev = 64;
std::mutex g_setup_mu;
int* g_scratch_ptr[kMaxDev] = {};  // device address of g_colour_scratch, per device

// once per device, with that device current: the device address of the
// scratch array (its host-side name is only a stand-in) and the kernel's
// shared-memory limit (the same constant amg_setup sets, so neither lowers it
// for the other).  The address is kept for the life of the process: after a
// cudaDeviceReset the library's module is loaded again and the kept address
// is stale, so the entry point must not be used after a reset.
int scratch_for_current_device(int** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return BAMG_ECUDA;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_colour_scratch) != cudaSuccess || !p) return BAMG_ECUDA;
        if (cudaFuncSetAttribute(colour_worklist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kWorklistSmemMax) != cudaSuccess)
            return BAMG_ECUDA;
        g_scratch_ptr[dev] = static_cast<int*>(p);
    }
    *out = g_scratch_ptr[dev];
    return BAMG_OK;
}

// n_colours = colour count, or -1 when the kernel reported a failure
__global__ void publish_count_kernel(const int* __restrict__ res, int* __restrict__ n_colours) {
    if (threadIdx.x == 0 && blockIdx.x == 0) n_colours[0] = res[1] ? -1 : res[0];
}

}  // namespace
}  // namespace bamg

using namespace bamg;

extern "C" int amg_colour_noalloc(const int* row_ptr, const int* col_idx, int n_nodes, int* colour, int* n_colours,
                                  void* stream) {
    if (!row_ptr || !col_idx || !colour || !n_colours || n_nodes < 1) return BAMG_EINVAL;
    if (n_nodes > kWorklistMaxNodes) return BAMG_EUNSUPPORTED;
    int* scratch = nullptr;
    const int st = scratch_for_current_device(&scratch);
    if (st != BAMG_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* qa = scratch;
    int* qb = scratch + kWorklistMaxNodes;
    int* res = scratch + 2 * kWorklistMaxNodes;  // [0] colours, [1] failure, [2] pattern check
    const size_t smem = (size_t)n_nodes * 5 + 16;
    // the worklist rule needs a valid, structurally symmetric pattern: check
    // it on the whole GPU first (the flag starts at zero on every call)
    if (cudaMemsetAsync(res + 2, 0, sizeof(int), s) != cudaSuccess) return BAMG_ECUDA;
    const int st_chk = launch_check_pattern(n_nodes, row_ptr, col_idx, nullptr, res + 2, s);
    if (st_chk != BAMG_OK) return st_chk;
    colour_worklist_kernel<<<1, 1024, smem, s>>>(n_nodes, row_ptr, col_idx, colour, qa, qb, res, res + 2);
    publish_count_kernel<<<1, 32, 0, s>>>(res, n_colours);
    return launched(2);
}
