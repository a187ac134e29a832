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
constexpr int ZK = 16;   // k chunk

// C = alpha op(A) op(B) + beta C with optional triangular structure (flags, see gw_internal.cuh):
// known-zero k ranges of a triangular operand are skipped, and with ZG_C_LOWER only tiles that
// reach the diagonal or below are computed (ZG_C_MIRROR also stores the conjugate transpose).
// ZT x ZT output tiles, (ZT/2)^2 threads with 2 x 2 outputs each.  The FP64 pipe, not shared
// memory, bounds this kernel; ZT = 16 gives four times as many CTAs for the small and triangular
// products of the inverse, whose few 32-wide tiles left most SMs idle.
template <int ZT>
__global__ void __launch_bounds__((ZT / 2) * (ZT / 2))
    zgemm_kernel(int M, int N, int K, double2 alpha, const double2 *__restrict__ A, int lda, int opA,
                 const double2 *__restrict__ B, int ldb, int opB, double2 beta, double2 *__restrict__ C, int ldc,
                 int flags)
{
    constexpr int H = ZT / 2, NT = H * H;
    __shared__ double2 As[ZK][ZT + 1];
    __shared__ double2 Bs[ZK][ZT + 1];
    const int i0 = blockIdx.y * ZT, j0 = blockIdx.x * ZT;
    if ((flags & ZG_C_LOWER) && j0 > i0 + ZT - 1)
        return;  // tile strictly above the diagonal
    const int tx = threadIdx.x % H, ty = threadIdx.x / H;
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
        for (int t = threadIdx.x; t < ZK * ZT; t += NT) {
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
            const double2 a0 = As[kk][ty], a1 = As[kk][ty + H];
            const double2 b0 = Bs[kk][tx], b1 = Bs[kk][tx + H];
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
            const int gi = i0 + ty + H * a, gj = j0 + tx + H * b;
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
// upper triangle is zeroed) and write Linv = L^-1 (lower, zero above) to Linv.
//
// One warp per block.  The FP64 pipe of an SM retires about 1.7 DFMA per clock, so a whole-warp
// FP64 instruction costs ~19 clocks whether or not its lanes are masked.  Both phases therefore
// spread the entries that are active at each step evenly over the 32 lanes, instead of giving each
// lane a fixed row:
//  * factorisation, pivot j: the entries (i, l) with j < l <= i are a prefix of a list ordered by
//    column l descending, so lane t takes list entries t, t + 32, ...;
//  * inverse, step i (forward substitution on the columns of I): row i of X is scaled by
//    1/L_ii, then the (k, c) entries with k > i, c <= i take X[k][c] -= L[k][i] X[i][c].
__global__ void __launch_bounds__(32)
    chol_diag_kernel(double2 *__restrict__ A, int lda, int n, double2 *__restrict__ Linv, int ldl, int pivot0,
                     uint32_t *err)
{
    __shared__ double2 S[32][33];
    __shared__ double2 X[32][33];
    __shared__ unsigned short ent[528];
    __shared__ double rd[32];
    const int lane = threadIdx.x;
    const unsigned FULL = 0xffffffffu;
    for (int t = lane; t < 32 * 32; t += 32) {
        const int i = t >> 5, l = t & 31;
        S[i][l] = (i < n && l < n && l <= i) ? A[(size_t)i * lda + l] : make_double2(0.0, 0.0);
        X[i][l] = make_double2(i == l && i < n ? 1.0 : 0.0, 0.0);
        if (l >= 1 && l <= i)  // position of (i, l): all entries of the columns right of l come first
            ent[(31 - l) * (32 - l) / 2 + (i - l)] = (unsigned short)((i << 8) | l);
    }
    __syncwarp(FULL);
    bool bad = false;
    for (int j = 0; j < n; ++j) {
        const double d = S[j][j].x;
        const bool ok = d > 0.0 && isfinite(d);
        const double y = ok ? rsqrt_newton(d) : 1.0;
        if (!ok && !bad && lane == 0)
            record_error(err, GW_E_NUMERIC, SITE_CHOL_PIVOT, (uint32_t)(pivot0 + j));
        bad = bad || !ok;
        __syncwarp(FULL);  // every lane has read the pivot before it is overwritten
        if (lane == j)
            S[j][j] = make_double2(ok ? d * y : 1.0, 0.0);
        else if (lane > j && lane < n)
            S[lane][j] = make_double2(S[lane][j].x * y, S[lane][j].y * y);
        if (lane == 0)
            rd[j] = y;
        __syncwarp(FULL);
        // S[i][l] -= S[i][j] conj(S[l][j]) for j < l <= i
        const int cnt = (31 - j) * (32 - j) / 2;
        for (int p = lane; p < cnt; p += 32) {
            const int e = ent[p], i = e >> 8, l = e & 255;
            const double2 a = S[i][j], b = S[l][j];
            double2 v = S[i][l];
            v.x = fma(-a.x, b.x, fma(-a.y, b.y, v.x));
            v.y = fma(-a.y, b.x, fma(a.x, b.y, v.y));
            S[i][l] = v;
        }
        __syncwarp(FULL);
    }
    for (int i = 0; i < n; ++i) {
        if (lane <= i)
            X[i][lane] = make_double2(X[i][lane].x * rd[i], X[i][lane].y * rd[i]);
        __syncwarp(FULL);
        const int w = i + 1, cnt = (n - 1 - i) * w;
        for (int p = lane; p < cnt; p += 32) {
            const int k = i + 1 + p / w, c = p - (p / w) * w;
            const double2 a = S[k][i], b = X[i][c];
            double2 v = X[k][c];
            v.x = fma(-a.x, b.x, fma(a.y, b.y, v.x));
            v.y = fma(-a.x, b.y, fma(-a.y, b.x, v.y));
            X[k][c] = v;
        }
        __syncwarp(FULL);
    }
    for (int t = lane; t < n * n; t += 32) {
        const int i = t / n, j = t % n;
        A[(size_t)i * lda + j] = j <= i ? S[i][j] : make_double2(0.0, 0.0);
        Linv[(size_t)i * ldl + j] = j <= i ? X[i][j] : make_double2(0.0, 0.0);
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
    // 32-wide tiles only when they alone make two full waves on 152 SMs
    const long t32 = (long)((N + 31) / 32) * ((M + 31) / 32) / ((flags & ZG_C_LOWER) ? 2 : 1);
    if (t32 >= 2 * 152) {
        dim3 grid((N + 31) / 32, (M + 31) / 32);
        zgemm_kernel<32><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, opA, B, ldb, opB, beta, C, ldc, flags);
    } else {
        dim3 grid((N + 15) / 16, (M + 15) / 16);
        zgemm_kernel<16><<<grid, 64, 0, s>>>(M, N, K, alpha, A, lda, opA, B, ldb, opB, beta, C, ldc, flags);
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_chol_diag(double2 *A, int lda, int n, double2 *Linv, int ldl, int pivot0, uint32_t *err,
                             cudaStream_t s)
{
    chol_diag_kernel<<<1, 32, 0, s>>>(A, lda, n, Linv, ldl, pivot0, err);
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
