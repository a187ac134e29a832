// Pair densities f_vc(r) = conj(psi_v(r)) psi_c(r) sqrt(2/(E_c - E_v))  -- Eq. (fdef), q = 0 --
// written straight into the operand layout of the rank-k update, plus the small load-time
// kernels (state transpose, FP64 weights, input checks).
#include "gw_internal.cuh"
#include "ptx.cuh"

namespace gw {

namespace {

constexpr int TPB = 256;

int grid_for(size_t n, int tpb = TPB)
{
    size_t g = (n + tpb - 1) / tpb;
    const size_t cap = 152 * 16;  // grid-stride beyond 16 CTAs per SM
    if (g > cap)
        g = cap;
    if (g < 1)
        g = 1;
    return static_cast<int>(g);
}

// psi [nb][nr] -> psiT [nr][nb] through 32x32 shared tiles (both sides coalesced).
__global__ void transpose_states_kernel(const float2 *__restrict__ psi, int nb, int nr, float2 *__restrict__ psiT)
{
    __shared__ float2 tile[32][33];
    const int r0 = blockIdx.x * 32, n0 = blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int n = n0 + dy, r = r0 + threadIdx.x;
        if (n < nb && r < nr)
            tile[dy][threadIdx.x] = psi[(size_t)n * nr + r];
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int r = r0 + dy, n = n0 + threadIdx.x;
        if (n < nb && r < nr)
            psiT[(size_t)r * nb + n] = tile[threadIdx.x][dy];
    }
}

__global__ void c128_to_c64_kernel(const double2 *__restrict__ in, size_t n, float2 *__restrict__ out)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = make_float2(static_cast<float>(in[i].x), static_cast<float>(in[i].y));
}

__global__ void check_finite_kernel(const float2 *__restrict__ x, size_t n, uint32_t *err)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 v = x[i];
        if (!isfinite(v.x) || !isfinite(v.y)) {
            record_error(err, GW_E_INVALID, SITE_INPUT, 0);
            return;
        }
    }
}

// sw[v][c] = sqrt(2 / (E_c - E_v)), differences and root in FP64 (energies in Hartree).
__global__ void weights_kernel(const double *__restrict__ E, int nv, int nc, float *__restrict__ sw)
{
    const int n = nv * nc;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int v = i / nc, c = i - v * nc;
        sw[i] = static_cast<float>(sqrt(2.0 / (E[nv + c] - E[v])));
    }
}

__device__ __forceinline__ float2 pair_value(const float2 *__restrict__ psiT, const float *__restrict__ sw, int r,
                                             int k, int nr, int nb, int nv, int nc)
{
    if (r >= nr || k >= nv * nc)
        return make_float2(0.f, 0.f);
    const int v = k / nc, c = k - v * nc;
    const float2 a = psiT[(size_t)r * nb + v];       // psi_v(r)
    const float2 b = psiT[(size_t)r * nb + nv + c];  // psi_c(r)
    const float s = sw[k];
    // conj(a) * b
    const float re = fmaf(a.x, b.x, a.y * b.y);
    const float im = fmaf(a.x, b.y, -a.y * b.x);
    return make_float2(re * s, im * s);
}

// Tiled TF32 planes.  One thread per (chunk, r, k-in-chunk), enumerated in the order the
// planes are stored so every warp writes 128 contiguous bytes per plane.
template <int NPL>
__global__ void pair_density_tf32_kernel(const float2 *__restrict__ psiT, const float *__restrict__ sw, int nr,
                                         int nb, int nv, int nc, int kpad, int nr_pad, float *__restrict__ F)
{
    const size_t per_chunk = (size_t)nr_pad * HERK_KC;
    const size_t total = (size_t)(kpad / HERK_KC) * per_chunk;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t kc = i / per_chunk;
        const int rem = static_cast<int>(i - kc * per_chunk);
        const int r8 = rem >> 6;             // 8-row group
        const int w = rem & 63;
        const int k4 = w >> 5;               // which 16-byte half of the 8-wide chunk
        const int rr = (w & 31) >> 2;        // row inside the group
        const int e = w & 3;                 // element inside the 16-byte core-matrix row
        const int r = r8 * 8 + rr;
        const int k = static_cast<int>(kc) * HERK_KC + k4 * 4 + e;
        const float2 f = pair_value(psiT, sw, r, k, nr, nb, nv, nc);
        float *base = F + kc * NPL * per_chunk + rem;
        if (NPL == 4) {
            const float rh = to_tf32(f.x), ih = to_tf32(f.y);
            base[0] = rh;
            base[per_chunk] = to_tf32(f.x - rh);
            base[2 * per_chunk] = ih;
            base[3 * per_chunk] = to_tf32(f.y - ih);
        } else {
            base[0] = to_tf32(f.x);
            base[per_chunk] = to_tf32(f.y);
        }
    }
}

// Plain complex64 f, [kpad][nr_pad] with r contiguous (operand of the CUDA-core update).
__global__ void pair_density_plain_kernel(const float2 *__restrict__ psiT, const float *__restrict__ sw, int nr,
                                          int nb, int nv, int nc, int kpad, int nr_pad, float2 *__restrict__ F)
{
    const size_t total = (size_t)kpad * nr_pad;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int k = static_cast<int>(i / nr_pad);
        const int r = static_cast<int>(i - (size_t)k * nr_pad);
        F[i] = pair_value(psiT, sw, r, k, nr, nb, nv, nc);
    }
}

// Plain complex64 f [rows][nr_pad] by 32 x 32 tiles: threads along k read 32 consecutive psi_c(r)
// of one r (psiT rows hold every state of one grid point), the tile is transposed in shared
// memory, and rows of F are written with r contiguous.
__global__ void __launch_bounds__(256) pair_density_tiled_kernel(const float2 *__restrict__ psiT,
                                                                 const float *__restrict__ sw, int nr, int nb, int nv,
                                                                 int nc, int rows, int nr_pad,
                                                                 float2 *__restrict__ F)
{
    __shared__ float2 T[32][33];
    const int k0 = blockIdx.y * 32, r0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    const int k = k0 + tx;
    const bool kin = k < nv * nc;
    const int v = kin ? k / nc : 0, c = kin ? k - v * nc : 0;
    const float w = kin ? sw[k] : 0.f;
    for (int dy = ty; dy < 32; dy += 8) {
        const int r = r0 + dy;
        float2 f = make_float2(0.f, 0.f);
        if (kin && r < nr) {
            const float2 a = psiT[(size_t)r * nb + v];
            const float2 b = psiT[(size_t)r * nb + nv + c];
            f = make_float2(fmaf(a.x, b.x, a.y * b.y) * w, fmaf(a.x, b.y, -a.y * b.x) * w);  // conj(a) b
        }
        T[dy][tx] = f;
    }
    __syncthreads();
    for (int dy = ty; dy < 32; dy += 8) {
        const int kk = k0 + dy, r = r0 + tx;
        if (kk < rows && r < nr_pad)
            F[(size_t)kk * nr_pad + r] = T[tx][dy];
    }
}

}  // namespace

cudaError_t launch_pair_density_rows(const float2 *psiT, const float *sw, int nr, int nb, int nv, int nc, int rows,
                                     int nr_pad, float2 *F, cudaStream_t s)
{
    dim3 grid((nr_pad + 31) / 32, (rows + 31) / 32);
    pair_density_tiled_kernel<<<grid, 256, 0, s>>>(psiT, sw, nr, nb, nv, nc, rows, nr_pad, F);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_transpose_states(const float2 *psi, int nb, int nr, float2 *psiT, cudaStream_t s)
{
    dim3 grid((nr + 31) / 32, (nb + 31) / 32), block(32, 8);
    transpose_states_kernel<<<grid, block, 0, s>>>(psi, nb, nr, psiT);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_c128_to_c64(const double2 *in, size_t n, float2 *out, cudaStream_t s)
{
    c128_to_c64_kernel<<<grid_for(n), TPB, 0, s>>>(in, n, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const float2 *x, size_t n, uint32_t *err, cudaStream_t s)
{
    check_finite_kernel<<<grid_for(n), TPB, 0, s>>>(x, n, err);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_weights(const double *E, int nv, int nc, float *sw, cudaStream_t s)
{
    weights_kernel<<<grid_for((size_t)nv * nc), TPB, 0, s>>>(E, nv, nc, sw);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pair_density(const float2 *psiT, const float *sw, int nr, int nb, int nv, int nc, int kpad,
                                int nr_pad, int prec, float *F, cudaStream_t s)
{
    const size_t total = (size_t)kpad * nr_pad;
    if (prec == GW_PREC_TF32X3)
        pair_density_tf32_kernel<4><<<grid_for(total), TPB, 0, s>>>(psiT, sw, nr, nb, nv, nc, kpad, nr_pad, F);
    else if (prec == GW_PREC_TF32X1)
        pair_density_tf32_kernel<2><<<grid_for(total), TPB, 0, s>>>(psiT, sw, nr, nb, nv, nc, kpad, nr_pad, F);
    else
        pair_density_plain_kernel<<<grid_for(total), TPB, 0, s>>>(psiT, sw, nr, nb, nv, nc, kpad, nr_pad,
                                                                  reinterpret_cast<float2 *>(F));
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gw
