// Row transforms to the G sphere (the two FFT phases of Sec. 4.1, pruned to the sphere).
//
// For every input row x(r), r = (j1 n2 + j2) n3 + j3, the kernel produces
//     y(G) = sum_r x(r) exp(+2 pi i (m1 j1/n1 + m2 j2/n2 + m3 j3/n3))   for G = m in the sphere,
// one axis at a time, keeping only what the sphere needs:
//     stage 1 (j3 -> m3):  the c3 distinct m3 values of the sphere,
//     stage 2 (j2 -> m2):  the cd distinct (m2, m3) pairs (a disk),
//     stage 3 (j1 -> m1):  the N_g sphere points.
// Input rows stream through shared memory one j1-plane at a time (coalesced loads); stages 1
// and 2 run per plane and stage 3 once per row.  Twiddles are FP64-derived tables
// exp(+2 pi i t/n) and indices advance incrementally (no integer division in the inner loops).
//
// The path applies it twice: to the rows of P (P is Hermitian, so the conjugate of a row
// transform with exp(+iG.r) is the column transform with exp(-iG.r)), and, after a conjugate
// transpose, to the rows of that intermediate, which yields P~(G, G').
#include "gw_internal.cuh"

namespace gw {

namespace {

struct SmemLayout {
    size_t tw, m3, disk, gmap, X, A1, A2, total;
};

__host__ __device__ inline size_t align16(size_t x)
{
    return (x + 15) & ~(size_t)15;
}

__host__ __device__ inline SmemLayout layout_for(const int n[3], int ng, int c3, int cd, int R)
{
    SmemLayout L;
    size_t o = 0;
    L.tw = o;
    o = align16(o + sizeof(float2) * (n[0] + n[1] + n[2]));
    L.m3 = o;
    o = align16(o + sizeof(int) * c3);
    L.disk = o;
    o = align16(o + sizeof(int) * 2 * cd);
    L.gmap = o;
    o = align16(o + sizeof(int) * 2 * ng);
    L.X = o;
    o = align16(o + sizeof(float2) * R * n[1] * n[2]);
    L.A1 = o;
    o = align16(o + sizeof(float2) * R * n[1] * c3);
    L.A2 = o;
    o = align16(o + sizeof(float2) * R * n[0] * cd);
    L.total = o;
    return L;
}

__device__ __forceinline__ void cmac(float2 &acc, float2 x, float2 w)
{
    acc.x = fmaf(x.x, w.x, fmaf(-x.y, w.y, acc.x));
    acc.y = fmaf(x.x, w.y, fmaf(x.y, w.x, acc.y));
}

__global__ void __launch_bounds__(256)
    dft_rows_kernel(const float2 *__restrict__ X, long long ldx, int rows, float2 *__restrict__ Y, long long ldy,
                    int n1, int n2, int n3, int ng, int c3, int cd, const int *__restrict__ g_m3,
                    const int *__restrict__ g_disk, const int *__restrict__ g_gmap, const float2 *__restrict__ g_tw,
                    int R)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int nn[3] = {n1, n2, n3};
    const SmemLayout L = layout_for(nn, ng, c3, cd, R);
    float2 *tw = reinterpret_cast<float2 *>(smem + L.tw);  // [n1 | n2 | n3]
    int *m3 = reinterpret_cast<int *>(smem + L.m3);
    int *disk = reinterpret_cast<int *>(smem + L.disk);
    int *gmap = reinterpret_cast<int *>(smem + L.gmap);
    float2 *Xs = reinterpret_cast<float2 *>(smem + L.X);
    float2 *A1 = reinterpret_cast<float2 *>(smem + L.A1);
    float2 *A2 = reinterpret_cast<float2 *>(smem + L.A2);
    const float2 *tw1 = tw, *tw2 = tw + n1, *tw3 = tw + n1 + n2;

    const int tid = threadIdx.x, nt = blockDim.x;
    for (int t = tid; t < n1 + n2 + n3; t += nt)
        tw[t] = g_tw[t];
    for (int t = tid; t < c3; t += nt)
        m3[t] = g_m3[t];
    for (int t = tid; t < 2 * cd; t += nt)
        disk[t] = g_disk[t];
    for (int t = tid; t < 2 * ng; t += nt)
        gmap[t] = g_gmap[t];

    const int row0 = blockIdx.x * R;
    const int plane = n2 * n3;
    for (int j1 = 0; j1 < n1; ++j1) {
        __syncthreads();
        // plane j1 of R rows -> shared (zero for rows past the end)
        for (int t = tid; t < R * plane; t += nt) {
            const int rho = t / plane, q = t - rho * plane;
            const int row = row0 + rho;
            Xs[t] = row < rows ? X[(size_t)row * ldx + (size_t)j1 * plane + q] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        // stage 1: A1[rho][j2][i3] = sum_j3 X[rho][j2][j3] e(m3 j3 / n3)
        for (int t = tid; t < R * n2 * c3; t += nt) {
            const int i3 = t % c3;
            const int rj = t / c3;  // rho * n2 + j2
            const float2 *x = Xs + (size_t)rj * n3;
            const int step = m3[i3];
            int idx = 0;
            float2 acc = make_float2(0.f, 0.f);
            for (int j3 = 0; j3 < n3; ++j3) {
                cmac(acc, x[j3], tw3[idx]);
                idx += step;
                if (idx >= n3)
                    idx -= n3;
            }
            A1[t] = acc;
        }
        __syncthreads();
        // stage 2: A2[rho][j1][d] = sum_j2 A1[rho][j2][i3(d)] e(m2(d) j2 / n2)
        for (int t = tid; t < R * cd; t += nt) {
            const int rho = t / cd, d = t - rho * cd;
            const int step = disk[2 * d], i3 = disk[2 * d + 1];
            const float2 *a = A1 + (size_t)rho * n2 * c3 + i3;
            int idx = 0;
            float2 acc = make_float2(0.f, 0.f);
            for (int j2 = 0; j2 < n2; ++j2) {
                cmac(acc, a[(size_t)j2 * c3], tw2[idx]);
                idx += step;
                if (idx >= n2)
                    idx -= n2;
            }
            A2[((size_t)rho * n1 + j1) * cd + d] = acc;
        }
    }
    __syncthreads();
    // stage 3: y[rho][g] = sum_j1 A2[rho][j1][d(g)] e(m1(g) j1 / n1)
    for (int t = tid; t < R * ng; t += nt) {
        const int rho = t / ng, g = t - rho * ng;
        const int row = row0 + rho;
        if (row >= rows)
            continue;
        const int step = gmap[2 * g], d = gmap[2 * g + 1];
        const float2 *a = A2 + (size_t)rho * n1 * cd + d;
        int idx = 0;
        float2 acc = make_float2(0.f, 0.f);
        for (int j1 = 0; j1 < n1; ++j1) {
            cmac(acc, a[(size_t)j1 * cd], tw1[idx]);
            idx += step;
            if (idx >= n1)
                idx -= n1;
        }
        Y[(size_t)row * ldy + g] = acc;
    }
}

// out[c][r] = conj(in[r][c]) for in of shape rows x cols.
__global__ void conj_transpose_kernel(const float2 *__restrict__ in, int rows, int cols, float2 *__restrict__ out)
{
    __shared__ float2 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int r = r0 + dy, c = c0 + threadIdx.x;
        if (r < rows && c < cols)
            tile[dy][threadIdx.x] = in[(size_t)r * cols + c];
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int c = c0 + dy, r = r0 + threadIdx.x;
        if (r < rows && c < cols) {
            const float2 v = tile[threadIdx.x][dy];
            out[(size_t)c * rows + r] = make_float2(v.x, -v.y);
        }
    }
}

// P~ is Hermitian in exact arithmetic; the two FP32 transforms leave a mismatch of rounding size
// between (G, G') and (G', G).  Replace P~ by its Hermitian part (P~ + P~^H) / 2, the nearest
// Hermitian matrix, so eps is exactly Hermitian and its Cholesky factor inverts all of it.
__global__ void hermitize_kernel(float2 *__restrict__ A, int n)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    const int g = blockIdx.y;
    if (h < g || h >= n)
        return;
    if (h == g) {
        A[(size_t)g * n + g].y = 0.f;
        return;
    }
    const float2 a = A[(size_t)g * n + h], b = A[(size_t)h * n + g];
    const float2 m = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
    A[(size_t)g * n + h] = m;
    A[(size_t)h * n + g] = make_float2(m.x, -m.y);
}

constexpr size_t DFT_SMEM_TARGET = 100 * 1024;
constexpr size_t DFT_SMEM_MAX = 220 * 1024;

int rows_per_cta(const DftPlan &p)
{
    for (int R = 8; R > 1; --R)
        if (layout_for(p.n, p.ng, p.c3, p.cd, R).total <= DFT_SMEM_TARGET)
            return R;
    return 1;
}

}  // namespace

size_t dft_smem_bytes(const DftPlan &p, int R)
{
    if (R <= 0)
        R = rows_per_cta(p);
    return layout_for(p.n, p.ng, p.c3, p.cd, R).total;
}

cudaError_t launch_dft_rows(const float2 *X, long long ldx, int rows, float2 *Y, long long ldy, const DftPlan &p,
                            cudaStream_t s)
{
    if (rows <= 0)
        return cudaSuccess;
    const int R = rows_per_cta(p);
    const size_t smem = layout_for(p.n, p.ng, p.c3, p.cd, R).total;
    if (smem > DFT_SMEM_MAX)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(dft_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    dft_rows_kernel<<<(rows + R - 1) / R, 256, smem, s>>>(X, ldx, rows, Y, ldy, p.n[0], p.n[1], p.n[2], p.ng, p.c3,
                                                          p.cd, p.m3list, p.disk, p.gmap, p.tw, R);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_hermitize(float2 *A, int n, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    dim3 grid((n + 255) / 256, n);
    hermitize_kernel<<<grid, 256, 0, s>>>(A, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_conj_transpose(const float2 *in, int rows, int cols, float2 *out, cudaStream_t s)
{
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
    conj_transpose_kernel<<<grid, block, 0, s>>>(in, rows, cols, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gw
