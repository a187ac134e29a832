// gw_eps_inv_noalloc: the FP64 Cholesky inverse of gw_eps_inv for callers that cannot allocate
// device memory.
//
// Who cannot allocate, and why:
//  * applications whose device memory is owned by another allocator (a framework's caching pool,
//    an arena sized at start-up): a raw cudaMalloc fragments that memory, or fails once the pool
//    has claimed it all;
//  * latency-sensitive loops: cudaFree synchronises the whole device, stalling every stream.
// This entry point therefore keeps its workspace in one file-scope static device array of a
// fixed maximum size, which every GPU that loads the library holds until the process exits.
// The call reads its status word back to the host and synchronises the given stream before it
// returns, so it blocks the calling thread until the inverse is done.
#include <mutex>

#include "gw_internal.cuh"

using namespace gw;

namespace {

constexpr int NOALLOC_MAX_N = 512;  // largest matrix order accepted
constexpr int NB = 32;              // Cholesky panel width (as in gw_eps_inv)
// A (N^2) | Y (N^2) | T (N^2) | W (N * NB) | diagonal-block inverses | one slot for the status word
constexpr size_t SCRATCH_ELEMS = 3ull * NOALLOC_MAX_N * NOALLOC_MAX_N + (size_t)NOALLOC_MAX_N * NB +
                                 (size_t)(NOALLOC_MAX_N / NB) * NB * NB + 1;

static __device__ __align__(256) double2 g_noalloc_scratch[SCRATCH_ELEMS];  // 12.9 MB per device

std::mutex g_mutex;
constexpr int MAX_DEVICES = 64;
double2 *g_scratch_ptr[MAX_DEVICES] = {};

// The host-side name of the array is only a stand-in: a kernel needs the device address, which
// is looked up once per device with that device current.
gw_status scratch_address(int device, double2 **out)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    if (device < 0 || device >= MAX_DEVICES)
        return GW_E_INVALID;
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return GW_E_CUDA;
        }
        g_scratch_ptr[device] = static_cast<double2 *>(p);
    }
    *out = g_scratch_ptr[device];
    return GW_OK;
}

#define NA_CUDA(call)                   \
    do {                                \
        if ((call) != cudaSuccess) {    \
            cudaGetLastError();         \
            return GW_E_CUDA;           \
        }                               \
    } while (0)

}  // namespace

extern "C" gw_status gw_eps_inv_noalloc(const void *eps, int n, void *epsinv, void *stream)
{
    if (!eps || !epsinv || n < 1)
        return GW_E_INVALID;
    if (n > NOALLOC_MAX_N)
        return GW_E_INVALID;  // the static workspace holds matrices of order <= 512
    int device = 0;
    NA_CUDA(cudaGetDevice(&device));
    // Both matrices must live on the current device: the kernels run there, and a pointer to
    // another GPU's memory would make them read or write that GPU's memory.
    for (const void *p : {eps, static_cast<const void *>(epsinv)}) {
        cudaPointerAttributes attr{};
        NA_CUDA(cudaPointerGetAttributes(&attr, p));
        if (attr.type != cudaMemoryTypeDevice || attr.device != device)
            return GW_E_INVALID;
    }
    double2 *base = nullptr;
    const gw_status st = scratch_address(device, &base);
    if (st != GW_OK)
        return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int N = n;
    double2 *A = base, *Y = A + (size_t)N * N, *T = Y + (size_t)N * N, *W = T + (size_t)N * N,
            *Dinv = W + (size_t)N * NB;
    uint32_t *status = reinterpret_cast<uint32_t *>(base + SCRATCH_ELEMS - 1);

    // The array keeps the previous call's contents: clear the status word (the enqueue clears Y).
    NA_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
    NA_CUDA(chol_inverse_enqueue(static_cast<const double2 *>(eps), N, static_cast<double2 *>(epsinv), A, Y, T, W,
                                 Dinv, status, s));
    uint32_t word = 0;
    NA_CUDA(cudaMemcpyAsync(&word, status, sizeof word, cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    if (word != 0)
        return static_cast<gw_status>(word & 0xFF);
    return GW_OK;
}
