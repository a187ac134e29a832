// gw_eps_inv_noalloc: the FP64 Cholesky inverse of gw_eps_inv for callers that cannot allocate
// device memory.
//
// Who cannot allocate, and why:
//  * code that runs while a stream is being captured into a CUDA graph: cudaMalloc and cudaFree
//    are not captured and would break or silently escape the graph;
//  * applications whose memory is owned by another allocator (a framework's caching pool, an
//    arena sized at start-up): a raw cudaMalloc fragments that memory or fails when the pool has
//    claimed it all;
//  * latency-sensitive loops: cudaFree synchronises the whole device.
// This entry point therefore keeps its workspace in one file-scope static device array of a
// fixed maximum size, which every GPU that loads the library holds until the process exits.
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
    double2 *base = nullptr;
    const gw_status st = scratch_address(device, &base);
    if (st != GW_OK)
        return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int N = n, nblk = (N + NB - 1) / NB;
    double2 *A = base, *Y = A + (size_t)N * N, *T = Y + (size_t)N * N, *W = T + (size_t)N * N,
            *Dinv = W + (size_t)N * NB;
    uint32_t *status = reinterpret_cast<uint32_t *>(base + SCRATCH_ELEMS - 1);
    const double2 one = make_double2(1, 0), zero = make_double2(0, 0), mone = make_double2(-1, 0);

    // The array keeps the previous call's contents: clear the status word and Y, copy the input.
    NA_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
    NA_CUDA(cudaMemcpyAsync(A, eps, (size_t)N * N * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    for (int kb = 0; kb < nblk; ++kb) {
        const int k0 = kb * NB, kn = std::min(NB, N - k0), rest = N - k0 - kn;
        double2 *Dk = Dinv + (size_t)kb * NB * NB;
        NA_CUDA(launch_chol_diag(A + (size_t)k0 * N + k0, N, kn, Dk, NB, k0, status, s));
        if (rest > 0) {
            double2 *panel = A + (size_t)(k0 + kn) * N + k0;
            NA_CUDA(launch_zgemm(rest, kn, kn, one, panel, N, 0, Dk, NB, 1, zero, W, NB, s));
            NA_CUDA(launch_copy_block(W, NB, panel, N, rest, kn, s));
            NA_CUDA(launch_zgemm(rest, rest, kn, mone, W, NB, 0, W, NB, 1, one, A + (size_t)(k0 + kn) * N + k0 + kn,
                                 N, s, ZG_C_LOWER));
        }
    }
    NA_CUDA(cudaMemsetAsync(Y, 0, (size_t)N * N * sizeof(double2), s));
    // Y = L^-1 by recursive halving (children before parents), leaves are the 32x32 inverses.
    struct Frame {
        int n0, n;
    };
    Frame order[2 * NOALLOC_MAX_N / NB + 8];
    int norder = 0;
    Frame stack[2 * NOALLOC_MAX_N / NB + 8];
    int nstack = 0;
    stack[nstack++] = {0, N};
    while (nstack > 0) {
        const Frame f = stack[--nstack];
        order[norder++] = f;
        if (f.n > NB) {
            const int n1 = std::max(NB, ((f.n / 2 + NB - 1) / NB) * NB);
            stack[nstack++] = {f.n0, n1};
            stack[nstack++] = {f.n0 + n1, f.n - n1};
        }
    }
    for (int i = norder - 1; i >= 0; --i) {
        const int n0 = order[i].n0, nn = order[i].n;
        if (nn <= NB) {
            NA_CUDA(launch_copy_block(Dinv + (size_t)(n0 / NB) * NB * NB, NB, Y + (size_t)n0 * N + n0, N, nn, nn, s));
            continue;
        }
        const int n1 = std::max(NB, ((nn / 2 + NB - 1) / NB) * NB), n2 = nn - n1;
        NA_CUDA(launch_zgemm(n2, n1, n1, one, A + (size_t)(n0 + n1) * N + n0, N, 0, Y + (size_t)n0 * N + n0, N, 0, zero,
                             T, n1, s, ZG_B_LOWER));
        NA_CUDA(launch_zgemm(n2, n1, n2, mone, Y + (size_t)(n0 + n1) * N + n0 + n1, N, 0, T, n1, 0, zero,
                             Y + (size_t)(n0 + n1) * N + n0, N, s, ZG_A_LOWER));
    }
    NA_CUDA(launch_zgemm(N, N, N, one, Y, N, 1, Y, N, 0, zero, static_cast<double2 *>(epsinv), N, s,
                         ZG_A_UPPER | ZG_B_LOWER | ZG_C_LOWER | ZG_C_MIRROR));
    uint32_t word = 0;
    NA_CUDA(cudaMemcpyAsync(&word, status, sizeof word, cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    if (word != 0)
        return static_cast<gw_status>(word & 0xFF);
    return GW_OK;
}
