// eps_GG' = delta_GG' - sqrt(V(G)) P~_GG' sqrt(V(G')) and its FP64 inverse (Sec. 5.1).
//
// The inverse is a blocked Cholesky eps = L L^H (right-looking, 32-wide panels) followed by
// eps^-1 = Y^H Y with Y = L^-1, assembled from one small kernel that factors and inverts a
// 32 x 32 diagonal block in shared memory and a complex128 GEMM kernel.  The same GEMM drives
// the paper's Newton iteration X <- X (2I - eps X) when that method is requested.
#include "gw_internal.cuh"

namespace gw {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ double2 cconj(double2 a)
{
    return make_double2(a.x, -a.y);
}

__global__ void eps_build_kernel(const float2 *__restrict__ PG, const double *__restrict__ sv, int ng,
                                 double2 *__restrict__ eps)
{
    const size_t n = (size_t)ng * ng;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int g = static_cast<int>(i / ng), h = static_cast<int>(i - (size_t)g * ng);
        const float2 p = PG[i];
        const double s = sv[g] * sv[h];
        eps[i] = make_double2((g == h ? 1.0 : 0.0) - s * (double)p.x, -s * (double)p.y);
    }
}

// ---------------------------------------------------------------------------- zgemm
constexpr int ZT = 32;   // output tile
constexpr int ZK = 16;   // k chunk

// C = alpha op(A) op(B) + beta C with optional triangular structure (flags, see gw_internal.cuh):
// known-zero k ranges of a triangular operand are skipped, and with ZG_C_LOWER only tiles that
// reach the diagonal or below are computed (ZG_C_MIRROR also stores the conjugate transpose).
__global__ void __launch_bounds__(256)
    zgemm_kernel(int M, int N, int K, double2 alpha, const double2 *__restrict__ A, int lda, int opA,
                 const double2 *__restrict__ B, int ldb, int opB, double2 beta, double2 *__restrict__ C, int ldc,
                 int flags)
{
    __shared__ double2 As[ZK][ZT + 1];
    __shared__ double2 Bs[ZK][ZT + 1];
    const int i0 = blockIdx.y * ZT, j0 = blockIdx.x * ZT;
    if ((flags & ZG_C_LOWER) && j0 > i0 + ZT - 1)
        return;  // tile strictly above the diagonal
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double2 acc[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
            acc[a][b] = make_double2(0.0, 0.0);
    int kbeg = 0;
    if (flags & ZG_B_LOWER)
        kbeg = max(kbeg, j0);  // op(B)[k][j] = 0 for k < j
    if (flags & ZG_A_UPPER)
        kbeg = max(kbeg, i0);  // op(A)[i][k] = 0 for k < i
    kbeg = (kbeg / ZK) * ZK;
    const int kend = (flags & ZG_A_LOWER) ? min(K, i0 + ZT) : K;  // op(A)[i][k] = 0 for k > i
    for (int k0 = kbeg; k0 < kend; k0 += ZK) {
        for (int t = threadIdx.x; t < ZK * ZT; t += 256) {
            int i, kk;
            if (opA == 0) {
                i = t / ZK;
                kk = t % ZK;
            } else {
                kk = t / ZT;
                i = t % ZT;
            }
            const int gi = i0 + i, gk = k0 + kk;
            double2 v = make_double2(0.0, 0.0);
            if (gi < M && gk < K)
                v = opA == 0 ? A[(size_t)gi * lda + gk] : cconj(A[(size_t)gk * lda + gi]);
            As[kk][i] = v;
            int j, kb;
            if (opB == 0) {
                kb = t / ZT;
                j = t % ZT;
            } else {
                j = t / ZK;
                kb = t % ZK;
            }
            const int gj = j0 + j, gk2 = k0 + kb;
            double2 w = make_double2(0.0, 0.0);
            if (gj < N && gk2 < K)
                w = opB == 0 ? B[(size_t)gk2 * ldb + gj] : cconj(B[(size_t)gj * ldb + gk2]);
            Bs[kb][j] = w;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < ZK; ++kk) {
            const double2 a0 = As[kk][ty], a1 = As[kk][ty + 16];
            const double2 b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
            acc[0][0].x = fma(a0.x, b0.x, fma(-a0.y, b0.y, acc[0][0].x));
            acc[0][0].y = fma(a0.x, b0.y, fma(a0.y, b0.x, acc[0][0].y));
            acc[0][1].x = fma(a0.x, b1.x, fma(-a0.y, b1.y, acc[0][1].x));
            acc[0][1].y = fma(a0.x, b1.y, fma(a0.y, b1.x, acc[0][1].y));
            acc[1][0].x = fma(a1.x, b0.x, fma(-a1.y, b0.y, acc[1][0].x));
            acc[1][0].y = fma(a1.x, b0.y, fma(a1.y, b0.x, acc[1][0].y));
            acc[1][1].x = fma(a1.x, b1.x, fma(-a1.y, b1.y, acc[1][1].x));
            acc[1][1].y = fma(a1.x, b1.y, fma(a1.y, b1.x, acc[1][1].y));
        }
        __syncthreads();
    }
    const bool use_beta = beta.x != 0.0 || beta.y != 0.0;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int gi = i0 + ty + 16 * a, gj = j0 + tx + 16 * b;
            if (gi < M && gj < N && (!(flags & ZG_C_LOWER) || gj <= gi)) {
                double2 v = cmul(alpha, acc[a][b]);
                if (use_beta) {
                    const double2 c = cmul(beta, C[(size_t)gi * ldc + gj]);
                    v.x += c.x;
                    v.y += c.y;
                }
                C[(size_t)gi * ldc + gj] = v;
                if ((flags & ZG_C_MIRROR) && gj < gi)
                    C[(size_t)gj * ldc + gi] = cconj(v);
            }
        }
}

// ---------------------------------------------------------------------------- diagonal block
// 1/sqrt(d) by the Newton-Raphson iteration y <- y (3 - d y^2) / 2 started from the FP32 estimate:
// each step doubles the number of correct bits (24 -> 48 -> FP64 rounding).  On this GPU an FP64
// FMA has a 64-cycle latency and a correctly rounded FP64 sqrt plus division cost more than 1000
// cycles, so two short Newton steps are the faster route to a pivot and its reciprocal.
__device__ __forceinline__ double rsqrt_newton(double d)
{
    const float df = static_cast<float>(d);
    if (!(df > 1e-30f) || !(df < 1e30f))
        return 1.0 / sqrt(d);
    double y = static_cast<double>(rsqrtf(df));
    const double hd = 0.5 * d;
    y = y * fma(-hd * y, y, 1.5);
    y = y * fma(-hd * y, y, 1.5);
    return y;
}

// Factor the n x n (n <= 32) Hermitian block A = L L^H in place (lower triangle; the strict
// upper triangle is zeroed) and write Linv = L^-1 (lower, zero above) to Linv.  The inverse is
// built row by row with each dot product split over eight lanes, so its critical path is 32
// short reductions rather than 32-term serial sums.
__global__ void __launch_bounds__(256)
    chol_diag_kernel(double2 *__restrict__ A, int lda, int n, double2 *__restrict__ Linv, int ldl, int pivot0,
                     uint32_t *err)
{
    __shared__ double2 S[32][33];
    __shared__ double2 T[32][33];
    __shared__ double rd[32];
    __shared__ int bad;
    const int tid = threadIdx.x;
    if (tid == 0)
        bad = 0;
    for (int t = tid; t < 32 * 32; t += blockDim.x) {
        const int i = t / 32, j = t % 32;
        S[i][j] = (i < n && j < n && j <= i) ? A[(size_t)i * lda + j] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (tid == 0) {
            const double d = S[j][j].x;
            double y;
            if (!(d > 0.0) || !isfinite(d)) {
                if (!bad)
                    record_error(err, GW_E_NUMERIC, SITE_CHOL_PIVOT, (uint32_t)(pivot0 + j));
                bad = 1;
                y = 1.0;
                S[j][j] = make_double2(1.0, 0.0);
            } else {
                y = rsqrt_newton(d);
                S[j][j] = make_double2(d * y, 0.0);
            }
            rd[j] = y;
        }
        __syncthreads();
        const double inv = rd[j];
        if (tid > j && tid < n) {
            S[tid][j].x *= inv;
            S[tid][j].y *= inv;
        }
        __syncthreads();
        // trailing update of the lower triangle: S[i][l] -= S[i][j] conj(S[l][j]), j < l <= i
        for (int t = tid; t < 32 * 32; t += blockDim.x) {
            const int i = t / 32, l = t % 32;
            if (i < n && l > j && l <= i) {
                const double2 p = cmul(S[i][j], cconj(S[l][j]));
                S[i][l].x -= p.x;
                S[i][l].y -= p.y;
            }
        }
        __syncthreads();
    }
    // L X = I row by row: X[i][c] = (delta_ic - sum_{c <= l < i} L[i][l] X[l][c]) / L[i][i].
    const int c = tid >> 3, part = tid & 7;
    for (int i = 0; i < n; ++i) {
        double2 s = make_double2(0.0, 0.0);
        if (c < i)
            for (int l = c + part; l < i; l += 8) {
                const double2 p = cmul(S[i][l], T[l][c]);
                s.x += p.x;
                s.y += p.y;
            }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
        }
        if (part == 0 && c < 32) {
            if (c > i)
                T[i][c] = make_double2(0.0, 0.0);
            else
                T[i][c] = make_double2(((c == i) ? 1.0 : 0.0) - s.x, -s.y);
        }
        __syncthreads();
        if (part == 0 && c <= i)
            T[i][c] = make_double2(T[i][c].x * rd[i], T[i][c].y * rd[i]);
        __syncthreads();
    }
    for (int t = tid; t < n * n; t += blockDim.x) {
        const int i = t / n, j = t % n;
        A[(size_t)i * lda + j] = j <= i ? S[i][j] : make_double2(0.0, 0.0);
        Linv[(size_t)i * ldl + j] = T[i][j];
    }
}

__global__ void copy_block_kernel(const double2 *__restrict__ src, int lds, double2 *__restrict__ dst, int ldd,
                                  int rows, int cols)
{
    const size_t n = (size_t)rows * cols;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const int i = static_cast<int>(t / cols), j = static_cast<int>(t - (size_t)i * cols);
        dst[(size_t)i * ldd + j] = src[(size_t)i * lds + j];
    }
}

__global__ void set_identity_kernel(double2 *A, int lda, int n, double scale)
{
    const size_t tot = (size_t)n * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
        const int i = static_cast<int>(t / n), j = static_cast<int>(t - (size_t)i * n);
        A[(size_t)i * lda + j] = make_double2(i == j ? scale : 0.0, 0.0);
    }
}

__global__ void two_minus_kernel(double2 *T, int n)
{
    const size_t tot = (size_t)n * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
        const int i = static_cast<int>(t / n), j = static_cast<int>(t - (size_t)i * n);
        double2 v = T[t];
        T[t] = make_double2((i == j ? 2.0 : 0.0) - v.x, -v.y);
    }
}

// X = A^H / den
__global__ void scaled_adjoint_kernel(const double2 *__restrict__ A, int n, const double *__restrict__ den,
                                      double2 *__restrict__ X)
{
    const double s = 1.0 / *den;
    const size_t tot = (size_t)n * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
        const int i = static_cast<int>(t / n), j = static_cast<int>(t - (size_t)i * n);
        const double2 a = A[(size_t)j * n + i];
        X[t] = make_double2(a.x * s, -a.y * s);
    }
}

// Single-CTA reductions (the matrices are at most a few thousand squared).
__global__ void max_absdiff_kernel(const double2 *__restrict__ A, const double2 *__restrict__ B, size_t n,
                                   double *out)
{
    __shared__ double red[256];
    double m = 0.0;
    for (size_t t = threadIdx.x; t < n; t += blockDim.x) {
        const double dx = A[t].x - B[t].x, dy = A[t].y - B[t].y;
        const double d = sqrt(dx * dx + dy * dy);
        m = d > m || d != d ? d : m;
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double o = red[threadIdx.x + s];
            red[threadIdx.x] = o > red[threadIdx.x] || o != o ? o : red[threadIdx.x];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        *out = red[0];
}

__global__ void row_abs_sum_max_kernel(const double2 *__restrict__ A, int n, double *out)
{
    __shared__ double red[256];
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) {
            const double2 a = A[(size_t)i * n + j];
            s += sqrt(a.x * a.x + a.y * a.y);
        }
        m = s > m ? s : m;
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            red[threadIdx.x] = red[threadIdx.x + s] > red[threadIdx.x] ? red[threadIdx.x + s] : red[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        *out = red[0];
}

int grid_for(size_t n)
{
    size_t g = (n + 255) / 256;
    if (g > 152 * 8)
        g = 152 * 8;
    return g < 1 ? 1 : static_cast<int>(g);
}

}  // namespace

cudaError_t launch_eps_build(const float2 *PG, const double *sv, int ng, double2 *eps, cudaStream_t s)
{
    eps_build_kernel<<<grid_for((size_t)ng * ng), 256, 0, s>>>(PG, sv, ng, eps);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_zgemm(int M, int N, int K, double2 alpha, const double2 *A, int lda, int opA, const double2 *B,
                         int ldb, int opB, double2 beta, double2 *C, int ldc, cudaStream_t s, int flags)
{
    if (M <= 0 || N <= 0)
        return cudaSuccess;
    dim3 grid((N + ZT - 1) / ZT, (M + ZT - 1) / ZT);
    zgemm_kernel<<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, opA, B, ldb, opB, beta, C, ldc, flags);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_chol_diag(double2 *A, int lda, int n, double2 *Linv, int ldl, int pivot0, uint32_t *err,
                             cudaStream_t s)
{
    chol_diag_kernel<<<1, 256, 0, s>>>(A, lda, n, Linv, ldl, pivot0, err);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_copy_block(const double2 *src, int lds, double2 *dst, int ldd, int rows, int cols,
                              cudaStream_t s)
{
    if (rows <= 0 || cols <= 0)
        return cudaSuccess;
    copy_block_kernel<<<grid_for((size_t)rows * cols), 256, 0, s>>>(src, lds, dst, ldd, rows, cols);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_set_identity(double2 *A, int lda, int n, double scale, cudaStream_t s)
{
    set_identity_kernel<<<grid_for((size_t)n * n), 256, 0, s>>>(A, lda, n, scale);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_two_minus(double2 *T, int n, cudaStream_t s)
{
    two_minus_kernel<<<grid_for((size_t)n * n), 256, 0, s>>>(T, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_scaled_adjoint(const double2 *A, int n, const double *d_den, double2 *X, cudaStream_t s)
{
    scaled_adjoint_kernel<<<grid_for((size_t)n * n), 256, 0, s>>>(A, n, d_den, X);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_max_absdiff(const double2 *A, const double2 *B, size_t n, double *out, cudaStream_t s)
{
    max_absdiff_kernel<<<1, 256, 0, s>>>(A, B, n, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_row_abs_sum_max(const double2 *A, int n, double *out, cudaStream_t s)
{
    row_abs_sum_max_kernel<<<1, 256, 0, s>>>(A, n, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gw
