// eps_GG' = delta_GG' - sqrt(V(G)) P~_GG' sqrt(V(G')) and its FP64 inverse (Sec. 5.1).
//
// The inverse is a blocked Cholesky eps = L L^H (right-looking, 32-wide panels) followed by
// eps^-1 = Y^H Y with Y = L^-1, assembled from one small kernel that factors and inverts a
// 32 x 32 diagonal block in shared memory and a complex128 GEMM kernel.  The same GEMM drives
// the paper's Newton iteration X <- X (2I - eps X) when that method is requested.
#include <algorithm>

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
constexpr int ZT = 16;    // output tile (ZT x ZT, one complex output per thread)
constexpr int ZKC = 32;   // k chunk staged in shared memory

// C = alpha op(A) op(B) + beta C with optional triangular structure (flags, see gw_internal.cuh):
// known-zero k ranges of a triangular operand are skipped, and with ZG_C_LOWER only tiles that
// reach the diagonal or below are computed (ZG_C_MIRROR also stores the conjugate transpose).
//
// FP64 on this GPU: each SM sub-partition retires about 0.42 lane-FMAs per clock, so one
// warp-wide DFMA holds its sub-partition for ~77 clocks and the kernel is bound by how many
// DFMAs each warp issues and on how many sub-partitions they run.  Each thread therefore owns a
// single output (4 DFMAs per k), a CTA is 8 warps (two per sub-partition) on a 16 x 16 tile, and
// even the small products of the factorisation spread over hundreds of warps.  Shared-memory and
// global traffic are minor next to that.  Batched products: problem blockIdx.z uses A + z sA,
// B + z sB, C + z sC.
__global__ void __launch_bounds__(256)
    zgemm_kernel(int M, int N, int K, double2 alpha, const double2 *__restrict__ A, int lda, int opA,
                 const double2 *__restrict__ B, int ldb, int opB, double2 beta, double2 *__restrict__ C, int ldc,
                 int flags, long sA, long sB, long sC)
{
    __shared__ double2 As[ZKC][ZT + 1];
    __shared__ double2 Bs[ZKC][ZT + 1];
    A += blockIdx.z * sA;
    B += blockIdx.z * sB;
    C += blockIdx.z * sC;
    const int i0 = blockIdx.y * ZT, j0 = blockIdx.x * ZT;
    if ((flags & ZG_C_LOWER) && j0 > i0 + ZT - 1)
        return;  // tile strictly above the diagonal
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    int kbeg = 0;
    if (flags & ZG_B_LOWER)
        kbeg = max(kbeg, j0);  // op(B)[k][j] = 0 for k < j
    if (flags & ZG_A_UPPER)
        kbeg = max(kbeg, i0);  // op(A)[i][k] = 0 for k < i
    const int kend = (flags & ZG_A_LOWER) ? min(K, i0 + ZT) : K;  // op(A)[i][k] = 0 for k > i
    double2 acc = make_double2(0.0, 0.0);
    for (int k0 = kbeg; k0 < kend; k0 += ZKC) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int t = tid + 256 * e;
            int i, kk;
            if (opA == 0) {
                i = t / ZKC;
                kk = t % ZKC;
            } else {
                kk = t / ZT;
                i = t % ZT;
            }
            const int gi = i0 + i, gk = k0 + kk;
            double2 v = make_double2(0.0, 0.0);
            if (gi < M && gk < kend)
                v = opA == 0 ? A[(size_t)gi * lda + gk] : cconj(A[(size_t)gk * lda + gi]);
            As[kk][i] = v;
            int j, kb;
            if (opB == 0) {
                kb = t / ZT;
                j = t % ZT;
            } else {
                j = t / ZKC;
                kb = t % ZKC;
            }
            const int gj = j0 + j, gk2 = k0 + kb;
            double2 w = make_double2(0.0, 0.0);
            if (gj < N && gk2 < kend)
                w = opB == 0 ? B[(size_t)gk2 * ldb + gj] : cconj(B[(size_t)gj * ldb + gk2]);
            Bs[kb][j] = w;
        }
        __syncthreads();
        const int kn = min(ZKC, kend - k0);
#pragma unroll 8
        for (int kk = 0; kk < kn; ++kk) {
            const double2 a = As[kk][ty], b = Bs[kk][tx];
            acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
            acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
        }
        __syncthreads();
    }
    const int gi = i0 + ty, gj = j0 + tx;
    if (gi < M && gj < N && (!(flags & ZG_C_LOWER) || gj <= gi)) {
        double2 v = cmul(alpha, acc);
        if (beta.x != 0.0 || beta.y != 0.0) {
            const double2 c = cmul(beta, C[(size_t)gi * ldc + gj]);
            v.x += c.x;
            v.y += c.y;
        }
        C[(size_t)gi * ldc + gj] = v;
        if ((flags & ZG_C_MIRROR) && gj < gi)
            C[(size_t)gj * ldc + gi] = cconj(v);
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

// 1/d by the Newton-Raphson iteration y <- y + y (1 - d y) from the FP32 reciprocal: each step
// doubles the number of correct bits (24 -> 48 -> FP64 rounding), two dependent FMAs per step.
__device__ __forceinline__ double rcp_newton(double d)
{
    const float df = static_cast<float>(d);
    if (!(fabsf(df) > 1e-30f) || !(fabsf(df) < 1e30f))
        return 1.0 / d;
    double y = static_cast<double>(__frcp_rn(df));
    y = fma(y, fma(-d, y, 1.0), y);
    y = fma(y, fma(-d, y, 1.0), y);
    return y;
}

// Factor the n x n (n <= 32) Hermitian block A = L L^H in place (lower triangle; the strict
// upper triangle is zeroed) and write Linv = L^-1 (lower, zero above) to Linv.
//
// The block is factored as A = L~ D L~^H (L~ unit lower, D real), and L = L~ D^1/2 is formed at
// the end.  The chain of dependent operations from one pivot to the next is then one reciprocal
// and one update; the square roots, the column scalings and the inverse of the unit-lower L~
// (no divisions) are off that chain or parallel over the block:
//  * pivot j (one barrier): the entries (i, l), j < l <= i, take S[i][l] -= S[i][j] conj(S[l][j]) r
//    with r = 1/d_j, column j left unscaled (it holds L~_ij d_j).  They are a prefix of a list
//    ordered by column l descending, at most 2 per thread.  The thread that updates (j+1, j+1)
//    forms the next reciprocal at once, so no other warp repeats it;
//  * L~_ij = S[i][j] r_j; X = L~^-1 by forward substitution on the columns of I, one entry
//    (k, c), k > i >= c, per thread and step;
//  * L = L~ diag(sqrt d), Linv = diag(1/sqrt d) X.
__global__ void __launch_bounds__(256)
    chol_diag_kernel(double2 *__restrict__ A, int lda, int n, double2 *__restrict__ Linv, int ldl, int pivot0,
                     uint32_t *err)
{
    __shared__ double2 S[32][33];
    __shared__ double2 X[32][33];
    __shared__ unsigned short ent[496];
    __shared__ double dv[32], rdv[32], qv[32];
    const int tid = threadIdx.x;
    for (int t = tid; t < 32 * 32; t += blockDim.x) {
        const int i = t >> 5, l = t & 31;
        S[i][l] = (i < n && l < n && l <= i) ? A[(size_t)i * lda + l] : make_double2(0.0, 0.0);
        X[i][l] = make_double2(i == l && i < n ? 1.0 : 0.0, 0.0);
        if (l >= 1 && l <= i)  // position of (i, l): all entries of the columns right of l come first
            ent[(31 - l) * (32 - l) / 2 + (i - l)] = (unsigned short)((i << 8) | l);
    }
    // pivot 0's reciprocal; every later one is formed by the thread that finishes its diagonal entry
    if (tid == 0 && n > 0) {
        const double d = S[0][0].x;
        const bool ok = d > 0.0 && isfinite(d);
        if (!ok)
            record_error(err, GW_E_NUMERIC, SITE_CHOL_PIVOT, (uint32_t)pivot0);
        dv[0] = ok ? d : 1.0;
        rdv[0] = ok ? rcp_newton(d) : 1.0;
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        const double r = rdv[j];
        const int cnt = (31 - j) * (32 - j) / 2;
        for (int p = tid; p < cnt; p += blockDim.x) {
            const int e = ent[p], i = e >> 8, l = e & 255;
            const double2 a = S[i][j], b = S[l][j];
            const double cx = a.x * r, cy = a.y * r;
            double2 v = S[i][l];
            v.x = fma(-cx, b.x, fma(-cy, b.y, v.x));
            v.y = fma(-cy, b.x, fma(cx, b.y, v.y));
            S[i][l] = v;
            if (i == j + 1 && l == j + 1 && l < n) {  // the next pivot is final: its reciprocal now
                const bool ok = v.x > 0.0 && isfinite(v.x);
                if (!ok)
                    record_error(err, GW_E_NUMERIC, SITE_CHOL_PIVOT, (uint32_t)(pivot0 + l));
                dv[l] = ok ? v.x : 1.0;
                rdv[l] = ok ? rcp_newton(v.x) : 1.0;
            }
        }
        __syncthreads();
    }
    // L~ in place below the diagonal; 1/sqrt(d) per column
    for (int t = tid; t < n * n; t += blockDim.x) {
        const int i = t / n, j = t % n;
        if (i > j)
            S[i][j] = make_double2(S[i][j].x * rdv[j], S[i][j].y * rdv[j]);
    }
    if (tid < n)
        qv[tid] = rsqrt_newton(dv[tid]);
    __syncthreads();
    for (int i = 0; i + 1 < n; ++i) {
        const int w = i + 1;
        if (tid < (n - 1 - i) * w) {
            const int k = i + 1 + tid / w, c = tid - (tid / w) * w;
            const double2 a = S[k][i], b = X[i][c];
            double2 v = X[k][c];
            v.x = fma(-a.x, b.x, fma(a.y, b.y, v.x));
            v.y = fma(-a.x, b.y, fma(-a.y, b.x, v.y));
            X[k][c] = v;
        }
        __syncthreads();
    }
    for (int t = tid; t < n * n; t += blockDim.x) {
        const int i = t / n, j = t % n;
        double2 l = make_double2(0.0, 0.0), x = make_double2(0.0, 0.0);
        if (j < i) {
            const double sq = dv[j] * qv[j];
            l = make_double2(S[i][j].x * sq, S[i][j].y * sq);
        } else if (j == i) {
            l = make_double2(dv[j] * qv[j], 0.0);
        }
        if (j <= i)
            x = make_double2(X[i][j].x * qv[i], X[i][j].y * qv[i]);
        A[(size_t)i * lda + j] = l;
        Linv[(size_t)i * ldl + j] = x;
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

// The nblk inverses of the 32x32 diagonal blocks (Dinv, leading dimension 32) onto the diagonal of
// Y (leading dimension N); blockIdx.x = block.
__global__ void scatter_diag_blocks_kernel(const double2 *__restrict__ Dinv, int N, double2 *__restrict__ Y)
{
    const int b = blockIdx.x, n0 = 32 * b, nb = min(32, N - n0);
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int i = t / nb, j = t % nb;
        Y[(size_t)(n0 + i) * N + n0 + j] = Dinv[(size_t)b * 32 * 32 + i * 32 + j];
    }
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
    return launch_zgemm_batched(M, N, K, alpha, A, lda, opA, 0, B, ldb, opB, 0, beta, C, ldc, 0, 1, s, flags);
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

cudaError_t launch_zgemm_batched(int M, int N, int K, double2 alpha, const double2 *A, int lda, int opA, long sA,
                                 const double2 *B, int ldb, int opB, long sB, double2 beta, double2 *C, int ldc,
                                 long sC, int batch, cudaStream_t s, int flags)
{
    if (M <= 0 || N <= 0 || batch <= 0)
        return cudaSuccess;
    dim3 grid((N + ZT - 1) / ZT, (M + ZT - 1) / ZT, batch);
    zgemm_kernel<<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, opA, B, ldb, opB, beta, C, ldc, flags, sA, sB, sC);
    count_launches(1);
    return cudaGetLastError();
}

// eps^-1 of a Hermitian positive-definite N x N complex128 matrix, in FP64 (Sec. 5.1 asks for the
// inverse; the factorisation route is this library's):
//  1. blocked right-looking Cholesky eps = L L^H with 32-wide panels; each diagonal block is
//     factored and inverted by chol_diag_kernel, the panel below it is solved as a product with
//     that inverse, and the trailing lower triangle takes the rank-32 update;
//  2. Y = L^-1 by recursive doubling: with the inverted blocks of size b on the diagonal of Y,
//     each pair of neighbours becomes one block of size 2b through
//     [L11 0; L21 L22]^-1 = [Y11 0; -Y22 L21 Y11  Y22],
//     and all pairs of one size go in one batched product (a trailing pair with a short second
//     block in one more);
//  3. eps^-1 = Y^H Y, lower half computed and mirrored.
// Workspace: A, Y, T (N^2 each), W (N x 32), Dinv (ceil(N/32) x 32 x 32).  Status words for a
// non-positive pivot go to err.
cudaError_t chol_inverse_enqueue(const double2 *eps, int N, double2 *epsinv, double2 *A, double2 *Y, double2 *T,
                                 double2 *W, double2 *Dinv, uint32_t *err, cudaStream_t s)
{
    constexpr int NB = 32;
    const int nblk = (N + NB - 1) / NB;
    const double2 one = make_double2(1, 0), zero = make_double2(0, 0), mone = make_double2(-1, 0);
    cudaError_t e;
#define ENQ(x)                         \
    do {                               \
        if ((e = (x)) != cudaSuccess)  \
            return e;                  \
    } while (0)
    ENQ(cudaMemcpyAsync(A, eps, (size_t)N * N * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    for (int kb = 0; kb < nblk; ++kb) {
        const int k0 = kb * NB, kn = std::min(NB, N - k0), rest = N - k0 - kn;
        double2 *Dk = Dinv + (size_t)kb * NB * NB;
        ENQ(launch_chol_diag(A + (size_t)k0 * N + k0, N, kn, Dk, NB, k0, err, s));
        if (rest > 0) {
            double2 *panel = A + (size_t)(k0 + kn) * N + k0;
            ENQ(launch_zgemm(rest, kn, kn, one, panel, N, 0, Dk, NB, 1, zero, W, NB, s));
            ENQ(launch_copy_block(W, NB, panel, N, rest, kn, s));
            // only the lower triangle of the trailing matrix is read later
            ENQ(launch_zgemm(rest, rest, kn, mone, W, NB, 0, W, NB, 1, one, A + (size_t)(k0 + kn) * N + k0 + kn, N,
                             s, ZG_C_LOWER));
        }
    }
    ENQ(cudaMemsetAsync(Y, 0, (size_t)N * N * sizeof(double2), s));
    scatter_diag_blocks_kernel<<<nblk, 256, 0, s>>>(Dinv, N, Y);
    count_launches(1);
    ENQ(cudaGetLastError());
    const long diag = (long)N + 1;
    for (int b = NB; b < N; b *= 2) {
        const int F = N / (2 * b);  // pairs of two full blocks
        if (F > 0) {
            // T_p = L21 Y11, then Y21 = -Y22 T_p, for the pairs starting at 2 p b
            ENQ(launch_zgemm_batched(b, b, b, one, A + (size_t)b * N, N, 0, 2 * b * diag, Y, N, 0, 2 * b * diag, zero,
                                     T, b, (long)b * b, F, s, ZG_B_LOWER));
            ENQ(launch_zgemm_batched(b, b, b, mone, Y + (size_t)b * diag, N, 0, 2 * b * diag, T, b, 0, (long)b * b,
                                     zero, Y + (size_t)b * N, N, 2 * b * diag, F, s, ZG_A_LOWER));
        }
        const int n0 = 2 * b * F, n2 = N - n0 - b;  // a last pair with a short second block
        if (n2 > 0) {
            ENQ(launch_zgemm(n2, b, b, one, A + (size_t)(n0 + b) * N + n0, N, 0, Y + (size_t)n0 * diag, N, 0, zero, T,
                             b, s, ZG_B_LOWER));
            ENQ(launch_zgemm(n2, b, n2, mone, Y + (size_t)(n0 + b) * diag, N, 0, T, b, 0, zero,
                             Y + (size_t)(n0 + b) * N + n0, N, s, ZG_A_LOWER));
        }
    }
    // (Y^H Y)[i][j] = sum_{k >= max(i, j)} conj(Y[k][i]) Y[k][j]; Hermitian, so the lower half is
    // computed and mirrored
    ENQ(launch_zgemm(N, N, N, one, Y, N, 1, Y, N, 0, zero, epsinv, N, s,
                     ZG_A_UPPER | ZG_B_LOWER | ZG_C_LOWER | ZG_C_MIRROR));
#undef ENQ
    return cudaSuccess;
}

}  // namespace gw
