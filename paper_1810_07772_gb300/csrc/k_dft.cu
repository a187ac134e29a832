// Row transforms to the G sphere (the two FFT phases of Sec. 4.1, pruned to the sphere).
//
// For every input row x(r), r = (j1 n2 + j2) n3 + j3, the kernel produces
//     y(G) = sum_r x(r) exp(+2 pi i (m1 j1/n1 + m2 j2/n2 + m3 j3/n3))   for G = m in the sphere,
// one axis at a time, keeping only what the sphere needs:
//     stage 1 (j3 -> m3):  the c3 distinct m3 values of the sphere,
//     stage 2 (j2 -> m2):  the cd distinct (m2, m3) pairs (a disk),
//     stage 3 (j1 -> m1):  the N_g sphere points.
// Input rows stream through shared memory one j1-plane at a time (coalesced loads); stages 1
// and 2 run per plane and stage 3 once per row.  Where the grid is a compiled size (square planes
// N <= 27, spheres at q = 0) the twiddles are compile-time constants that the FMAs take as
// immediate operands; elsewhere they are FP64-derived tables exp(+2 pi i t/n) with indices that
// advance incrementally (no integer division in the inner loops).
//
// The path applies it twice: to the rows of P (P is Hermitian, so the conjugate of a row
// transform with exp(+iG.r) is the column transform with exp(-iG.r)), and, after a conjugate
// transpose, to the rows of that intermediate, which yields P~(G, G').
#include <algorithm>
#include <utility>

#include "gw_internal.cuh"
#include "twiddle_const.cuh"

namespace gw {

namespace {

constexpr int DFT_THREADS = 256;
constexpr int GPT_MAX = 16;  // stage-3 outputs (row, G) per thread kept in registers, at most

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
    o = align16(o + sizeof(float2) * 2 * R * n[1] * n[2]);  // double-buffered j1-plane
    L.A1 = o;
    o = align16(o + sizeof(float2) * R * n[1] * c3);
    L.A2 = o;
    o = align16(o + sizeof(float2) * R * cd);  // current plane only
    L.total = o;
    return L;
}

__device__ __forceinline__ void cmac(float2 &acc, float2 x, float2 w)
{
    acc.x = fmaf(x.x, w.x, fmaf(-x.y, w.y, acc.x));
    acc.y = fmaf(x.x, w.y, fmaf(x.y, w.x, acc.y));
}

__device__ __forceinline__ void cp_async8(void *dst_smem, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(
                     dst_smem))),
                 "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(
                     dst_smem))),
                 "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// GPT (stage-3 outputs per thread) is sized to R N_g at launch: registers, not shared memory,
// decide how many CTAs share an SM, and every CTA more hides more of the barrier waits between
// the three stages.
template <int R, int GPT>
__global__ void __launch_bounds__(DFT_THREADS, GPT <= 12 ? 3 : 2)
    dft_rows_kernel(const float2 *__restrict__ X, long long ldx, int rows, float2 *__restrict__ Y, long long ldy,
                    int n1, int n2, int n3, int ng, int c3, int cd, const int *__restrict__ g_m3,
                    const int *__restrict__ g_disk, const int *__restrict__ g_gmap, const float2 *__restrict__ g_tw)
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

    const int tid = threadIdx.x;
    for (int t = tid; t < n1 + n2 + n3; t += DFT_THREADS)
        tw[t] = g_tw[t];
    for (int t = tid; t < c3; t += DFT_THREADS)
        m3[t] = g_m3[t];
    for (int t = tid; t < 2 * cd; t += DFT_THREADS)
        disk[t] = g_disk[t];
    for (int t = tid; t < 2 * ng; t += DFT_THREADS)
        gmap[t] = g_gmap[t];

    const int row0 = blockIdx.x * R;
    const int plane = n2 * n3;
    // plane j1 of the R rows -> Xs[buf] (asynchronous 8-byte copies; zeros past the last row)
    auto issue_plane = [&](int j1, int buf) {
        float2 *dst = Xs + (size_t)buf * R * plane;
        for (int t = tid; t < R * plane; t += DFT_THREADS) {
            const int rho = t / plane, q = t - rho * plane;
            const int row = row0 + rho;
            if (row < rows)
                cp_async8(dst + t, X + (size_t)row * ldx + (size_t)j1 * plane + q);
            else
                dst[t] = make_float2(0.f, 0.f);
        }
        cp_async_commit();
    };

    // stage-3 outputs owned by this thread: items u = tid + 256 * s over (rho, g)
    float2 acc3[GPT];
    int idx3[GPT];
#pragma unroll
    for (int s = 0; s < GPT; ++s) {
        acc3[s] = make_float2(0.f, 0.f);
        idx3[s] = 0;
    }
    const int n3items = R * ng;

    __syncthreads();  // tables visible
    issue_plane(0, 0);
    for (int j1 = 0; j1 < n1; ++j1) {
        const int buf = j1 & 1;
        if (j1 + 1 < n1) {
            issue_plane(j1 + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float2 *xb = Xs + (size_t)buf * R * plane;
        // stage 1: A1[rho][j2][i3] = sum_j3 X[rho][j2][j3] e(m3 j3 / n3).  Whole rounds of items take
        // all R rows (one twiddle serves R rows); the items left over after the last whole round go
        // one row each, so that round does not leave most threads waiting at the barrier.
        const int nfull = n2 * c3, whole = (nfull / DFT_THREADS) * DFT_THREADS;
        for (int t = tid; t < whole; t += DFT_THREADS) {
            const int j2 = t / c3, i3 = t - j2 * c3;
            const int step = m3[i3];
            float2 acc[R];
#pragma unroll
            for (int rho = 0; rho < R; ++rho)
                acc[rho] = make_float2(0.f, 0.f);
            int idx = 0;
            const float2 *x = xb + j2 * n3;
            for (int j3 = 0; j3 < n3; ++j3) {
                const float2 w = tw3[idx];
#pragma unroll
                for (int rho = 0; rho < R; ++rho)
                    cmac(acc[rho], x[rho * plane + j3], w);
                idx += step;
                if (idx >= n3)
                    idx -= n3;
            }
#pragma unroll
            for (int rho = 0; rho < R; ++rho)
                A1[(rho * n2 + j2) * c3 + i3] = acc[rho];
        }
        for (int t = tid; t < (nfull - whole) * R; t += DFT_THREADS) {
            const int item = whole + t / R, rho = t - (t / R) * R;
            const int j2 = item / c3, i3 = item - j2 * c3;
            const int step = m3[i3];
            float2 acc = make_float2(0.f, 0.f);
            int idx = 0;
            const float2 *x = xb + rho * plane + j2 * n3;
            for (int j3 = 0; j3 < n3; ++j3) {
                cmac(acc, x[j3], tw3[idx]);
                idx += step;
                if (idx >= n3)
                    idx -= n3;
            }
            A1[(rho * n2 + j2) * c3 + i3] = acc;
        }
        __syncthreads();
        // stage 2: A2[rho][d] = sum_j2 A1[rho][j2][i3(d)] e(m2(d) j2 / n2), one (row, d) per item:
        // the disk has about a hundred points, so items over rows keep more threads busy
        for (int t = tid; t < R * cd; t += DFT_THREADS) {
            const int rho = t / cd, d = t - rho * cd;
            const int step = disk[2 * d], i3 = disk[2 * d + 1];
            float2 acc = make_float2(0.f, 0.f);
            int idx = 0;
            const float2 *a1 = A1 + rho * n2 * c3 + i3;
            for (int j2 = 0; j2 < n2; ++j2) {
                cmac(acc, a1[j2 * c3], tw2[idx]);
                idx += step;
                if (idx >= n2)
                    idx -= n2;
            }
            A2[rho * cd + d] = acc;
        }
        __syncthreads();
        // stage 3 (this plane's term): y[rho][g] += A2[rho][d(g)] e(m1(g) j1 / n1)
#pragma unroll
        for (int s = 0; s < GPT; ++s) {
            const int u = tid + DFT_THREADS * s;
            if (u < n3items) {
                const int rho = u / ng, g = u - rho * ng;
                cmac(acc3[s], A2[rho * cd + gmap[2 * g + 1]], tw1[idx3[s]]);
                idx3[s] += gmap[2 * g];
                if (idx3[s] >= n1)
                    idx3[s] -= n1;
            }
        }
        // the next iteration's wait + __syncthreads orders these reads before A1/A2 are rewritten
    }
#pragma unroll
    for (int s = 0; s < GPT; ++s) {
        const int u = tid + DFT_THREADS * s;
        if (u < n3items) {
            const int rho = u / ng, g = u - rho * ng;
            const int row = row0 + rho;
            if (row < rows)
                Y[(size_t)row * ldy + g] = acc3[s];
        }
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

// ---------------------------------------------------------------------------------------------
// Two-kernel form.  Stages 1 and 2 of one (row, j1) plane are independent of every other plane, so
// one warp takes one plane at a time: it stages the n2 x n3 plane in its own shared memory,
// forms the c3 stage-1 lines and the cd stage-2 disk values with __syncwarp only, and writes
// the cd values to a workspace [rows][n1][cd].  A second kernel does stage 3 per row (one CTA
// per row: the row's n1 x cd values in shared memory, the N_g outputs over the threads).  The
// sums run in the same order with the same twiddles as in dft_rows_kernel.
//
// Stage 1 (two thirds of the work) takes one line j2 per lane when n3 is a compiled size: the n3
// inputs sit in registers and, output by output, every lane reads the same twiddle (one
// broadcast shared-memory access per complex FMA of each lane) where the per-output form read the
// input and the twiddle for every FMA.
//
// When the sphere's m3 values are exactly -M..M (every sphere |G|^2 < gcut is symmetric under
// G -> -G), stage 1 pairs the inputs j3 and n3 - j3: with s = x_j + x_{n-j}, t = x_j - x_{n-j} and
// e(m j / n) = c + i s_m,
//     sum_j x_j e(+-m j / n) = x_0 + (-1)^m x_{n/2} + sum_{0<j<n/2} s_j c  +-  i sum_{0<j<n/2} t_j s_m,
// so one cosine sum and one sine sum give the outputs m and -m: a quarter of the multiplies and
// twiddle reads of the plain sums.  The table's sine carries the sign of the exponent, so the
// same code serves both directions.  Stage 2 does the same over j2 for the disk points (m2, m3)
// and (-m2, m3) (the disk of a sphere is symmetric in m2): a1[j2] + a1[n2 - j2] and
// a1[j2] - a1[n2 - j2] are formed in place once per column, and one lane makes both outputs of
// a pair.  Sums run in another order than in dft_rows_kernel; both are FP32 sums of the same
// terms.
constexpr int P12_WARPS = 8;

// Per warp: a1 [n2][c3] and, for the generic stage 1 only, the plane [n2][n3 + 1] (rows padded:
// one lane per row reads them).  The compiled stage 1 (stage, even n3) copies the plane with
// coalesced 16-byte loads into [n2][p12_pitch(n3)] rows: a pitch of 2 mod 4 complex values (4 mod 8
// words) puts the 16-byte reads of eight lanes on eight different bank quadruples.  Pair-density
// rows form their products conj(psi_v) psi_c w during that copy.
__host__ __device__ constexpr int p12_pitch(int n3) { return n3 + 2 + ((n3 % 4 == 2) ? 2 : 0); }

__host__ __device__ inline size_t p12_warp_floats2(int n2, int n3, int c3, bool plane, bool stage = false)
{
    return (align16(sizeof(float2) * ((plane ? (size_t)n2 * (n3 + 1) : 0) + (size_t)n2 * c3)) +
            (stage ? sizeof(float2) * (size_t)n2 * p12_pitch(n3) : 0)) /
           sizeof(float2);
}

// Twiddle tables of the plane kernel, unrolled so the inner loops carry no index arithmetic:
// tw3m[i3][j3] = e(m3(i3) j3 / n3) and tw2d[d][j2] = e(m2(d) j2 / n2), the latter with rows of
// n2 + 1 so that lanes on neighbouring disk points hit different banks.  With stage-2 pairs
// (np2 > 0) tw2d is replaced by the pair list and tw2m[m2][j2] = e(m2 j2 / n2) for m2 <= k2,
// j2 <= n2 / 2, rows of p12_ld2 (odd) entries.
__host__ __device__ inline int p12_ld2(int n2) { return (n2 / 2 + 1) | 1; }

__host__ __device__ inline size_t p12_tables(const int n[3], int c3, int cd, int np2, int k2)
{
    const size_t t2 = np2 > 0 ? (size_t)np2 * 2 + (size_t)(k2 + 1) * p12_ld2(n[1]) : (size_t)cd * (n[1] + 1);
    return align16(sizeof(float2) * (size_t)c3 * n[2]) + align16(sizeof(float2) * t2);
}

__host__ __device__ inline size_t p12_smem(const int n[3], int c3, int cd, int np2, int k2, bool plane,
                                           bool stage = false)
{
    const size_t tables = align16(sizeof(float2) * (n[0] + n[1] + n[2]) + sizeof(int) * (c3 + 2 * cd));
    return tables + p12_tables(n, c3, cd, np2, k2) +
           P12_WARPS * p12_warp_floats2(n[1], n[2], c3, plane, stage) * sizeof(float2);
}

// Pair-density rows (PAIR): row k of the transform is f_k(r) = conj(psi_v(r)) psi_c(r) w_k with
// k = v nc + c (Eq. fdef), formed while the lines are loaded from the states psi [nb][N_r] (X,
// row stride ldx = N_r) instead of being read from a stored [k][N_r] array.  The products are
// written with the same FP32 operations as in pair_density_tiled_kernel.  Tasks then run
// j1-major, so the warps of a CTA share psi_v.
struct PairSrc {
    const float *sw;
    int nv, nc;
    int c0;  // state index of the first c (nv for the unoccupied states, 0 for all loaded states)
};

// The product times w is rounded on its own (__fmul_rn): where the caller adds it to something the
// compiler would otherwise contract the two into one FMA and round differently.
template <bool PAIR>
__device__ __forceinline__ float2 pair_or_x(float2 a, float2 b, float w)
{
    return PAIR ? make_float2(__fmul_rn(fmaf(a.x, b.x, a.y * b.y), w), __fmul_rn(fmaf(a.x, b.y, -a.y * b.x), w)) : a;
}

template <int N3, bool PAIR>  // N3 = 0: any n3 (one output per lane)
__global__ void __launch_bounds__(P12_WARPS * 32)
    dft_plane12_kernel(const float2 *__restrict__ X, long long ldx, int rows, int n1, int n2, int n3, int c3,
                       int sym3, int cd, const int *__restrict__ g_m3, const int *__restrict__ g_disk,
                       int np2, int k2, const int4 *__restrict__ g_pair2, const float2 *__restrict__ g_tw,
                       float2 *__restrict__ Y2, PairSrc ps)
{
    extern __shared__ __align__(16) uint8_t smem[];
    float2 *tw = reinterpret_cast<float2 *>(smem);  // [n1 | n2 | n3]
    int *m3 = reinterpret_cast<int *>(tw + n1 + n2 + n3);
    int *disk = m3 + c3;
    const int nn[3] = {n1, n2, n3};
    float2 *tw3m = reinterpret_cast<float2 *>(
        smem + align16(sizeof(float2) * (n1 + n2 + n3) + sizeof(int) * (c3 + 2 * cd)));
    float2 *tw2d = reinterpret_cast<float2 *>(reinterpret_cast<uint8_t *>(tw3m) + align16(sizeof(float2) * c3 * n3));
    int4 *pair2 = reinterpret_cast<int4 *>(tw2d);  // np2 > 0: [np2] (16-byte aligned), then tw2m
    const int ld2 = p12_ld2(n2), h2 = (n2 - 1) / 2;
    float2 *tw2m = tw2d + (size_t)np2 * 2;
    float2 *wbase =
        reinterpret_cast<float2 *>(reinterpret_cast<uint8_t *>(tw3m) + p12_tables(nn, c3, cd, np2, k2));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int t = tid; t < n1 + n2 + n3; t += blockDim.x)
        tw[t] = g_tw[t];
    for (int t = tid; t < c3; t += blockDim.x)
        m3[t] = g_m3[t];
    for (int t = tid; t < 2 * cd; t += blockDim.x)
        disk[t] = g_disk[t];
    __syncthreads();
    const float2 *tw2 = tw + n1, *tw3 = tw + n1 + n2;
    for (int t = tid; t < c3 * n3; t += blockDim.x) {
        const int i3 = t / n3, j3 = t - i3 * n3;
        tw3m[t] = tw3[(int)(((long long)m3[i3] * j3) % n3)];
    }
    if (np2 > 0) {
        for (int t = tid; t < np2; t += blockDim.x)
            pair2[t] = g_pair2[t];
        for (int t = tid; t < (k2 + 1) * ld2; t += blockDim.x) {
            const int m2 = t / ld2, j2 = t - m2 * ld2;
            tw2m[t] = tw2[(m2 * j2) % n2];
        }
    } else {
        for (int t = tid; t < cd * n2; t += blockDim.x) {
            const int d = t / n2, j2 = t - d * n2;
            tw2d[d * (n2 + 1) + j2] = tw2[(int)(((long long)disk[2 * d] * j2) % n2)];
        }
    }
    __syncthreads();
    const int plane = n2 * n3;
    constexpr bool kPlane = N3 == 0;
    constexpr bool kStage = N3 > 0 && N3 % 2 == 0;  // the plane (or pair product) staged in shared memory
    constexpr int SP = N3 > 0 ? p12_pitch(N3) : 1;
    float2 *xp = wbase + (size_t)warp * p12_warp_floats2(n2, n3, c3, kPlane, kStage);
    float2 *a1 = xp + (kPlane ? (size_t)n2 * (n3 + 1) : 0);
    float2 *pl = xp + align16(sizeof(float2) * ((kPlane ? (size_t)n2 * (n3 + 1) : 0) + (size_t)n2 * c3)) /
                          sizeof(float2);  // kStage: [n2][SP]
    const int ld3 = n3 + 1;
    // 16-byte loads of the lines need an even n3, an even row stride and an aligned base
    const bool vec = (N3 % 2 == 0) && (ldx % 2 == 0) && ((reinterpret_cast<size_t>(X) & 15) == 0);
    const long long ntasks = (long long)rows * n1;
    for (long long task = (long long)blockIdx.x * P12_WARPS + warp; task < ntasks;
         task += (long long)gridDim.x * P12_WARPS) {
        long long row;
        int j1;
        if (PAIR) {
            j1 = (int)(task / rows);
            row = task - (long long)j1 * rows;
        } else {
            row = task / n1;
            j1 = (int)(task - row * n1);
        }
        // PAIR: src is the plane of psi_c and srcv that of psi_v, w the weight of the pair
        const float2 *src, *srcv = nullptr;
        float w = 0.f;
        if (PAIR) {
            const int kk = (int)row, v = kk / ps.nc;
            src = X + (size_t)(ps.c0 + kk - v * ps.nc) * ldx + (size_t)j1 * plane;
            srcv = X + (size_t)v * ldx + (size_t)j1 * plane;
            w = ps.sw[kk];
        } else {
            src = X + row * ldx + (size_t)j1 * plane;
        }
        if (kPlane) {
            int j2 = lane / n3, j3 = lane - (lane / n3) * n3;  // q = lane + 32 i -> (j2, j3), no division in the loop
            const int dj2 = 32 / n3, dj3 = 32 - (32 / n3) * n3;
            for (int q = lane; q < plane; q += 32) {
                xp[j2 * ld3 + j3] = pair_or_x<PAIR>(PAIR ? srcv[q] : src[q], src[q], w);
                j2 += dj2;
                j3 += dj3;
                if (j3 >= n3) {
                    j3 -= n3;
                    ++j2;
                }
            }
        }
        if (kStage && vec) {
            // the whole plane with coalesced 16-byte loads (512 bytes per warp instruction) into
            // rows of SP complex values
            constexpr int QR = kStage ? N3 / 2 : 1;  // 16-byte words per line (the branch needs kStage)
            const float4 *s4 = reinterpret_cast<const float4 *>(src);
            const float4 *v4 = reinterpret_cast<const float4 *>(srcv);
#pragma unroll 4
            for (int q = lane; q < n2 * QR; q += 32) {
                const int j2 = q / QR, c = q - j2 * QR;
                float4 x = __ldg(s4 + q);
                if (PAIR) {  // x <- conj(psi_v) psi_c w
                    const float4 a = __ldg(v4 + q);
                    const float2 lo = pair_or_x<PAIR>(make_float2(a.x, a.y), make_float2(x.x, x.y), w);
                    const float2 hi = pair_or_x<PAIR>(make_float2(a.z, a.w), make_float2(x.z, x.w), w);
                    x = make_float4(lo.x, lo.y, hi.x, hi.y);
                }
                *reinterpret_cast<float4 *>(pl + j2 * SP + 2 * c) = x;
            }
        }
        __syncwarp();
        // stage 1: a1[j2][i3] = sum_j3 x[j2][j3] e(m3 j3 / n3)
        if (N3 > 0) {
            for (int j2 = lane; j2 < n2; j2 += 32) {
                float2 xr[N3 > 0 ? N3 : 1];
                const float2 *line = src + (size_t)j2 * N3;  // the line from global memory (L1 keeps it)
                if (kStage && vec) {
                    const float2 *ls = pl + j2 * SP;  // the staged line
#pragma unroll
                    for (int j3 = 0; j3 < N3; j3 += 2) {
                        const float4 v = *reinterpret_cast<const float4 *>(ls + j3);
                        xr[j3] = make_float2(v.x, v.y);
                        xr[j3 + 1 < N3 ? j3 + 1 : j3] = make_float2(v.z, v.w);
                    }
                } else if (vec) {
#pragma unroll
                    for (int j3 = 0; j3 < N3; j3 += 2) {
                        const float4 v = __ldg(reinterpret_cast<const float4 *>(line + j3));
                        xr[j3] = make_float2(v.x, v.y);
                        xr[j3 + 1 < N3 ? j3 + 1 : j3] = make_float2(v.z, v.w);
                    }
                    if (PAIR) {  // x <- conj(psi_v) psi_c w
                        const float2 *lv = srcv + (size_t)j2 * N3;
#pragma unroll
                        for (int j3 = 0; j3 < N3; j3 += 2) {
                            const float4 a = __ldg(reinterpret_cast<const float4 *>(lv + j3));
                            xr[j3] = pair_or_x<PAIR>(make_float2(a.x, a.y), xr[j3], w);
                            if (j3 + 1 < N3)
                                xr[j3 + 1] = pair_or_x<PAIR>(make_float2(a.z, a.w), xr[j3 + 1], w);
                        }
                    }
                } else {
#pragma unroll
                    for (int j3 = 0; j3 < N3; ++j3)
                        xr[j3] = pair_or_x<PAIR>(PAIR ? __ldg(srcv + (size_t)j2 * N3 + j3) : __ldg(line + j3),
                                                 __ldg(line + j3), w);
                }
                if (sym3 >= 0) {
                    constexpr int H = (N3 - 1) / 2;  // pairs (j, n3 - j), 0 < j < n3 / 2
                    float2 a0 = xr[0];
#pragma unroll
                    for (int j = 1; j <= H; ++j) {  // xr[j] <- s_j, xr[n3 - j] <- t_j
                        const float2 u = xr[j], v = xr[N3 - j];
                        xr[j] = make_float2(u.x + v.x, u.y + v.y);
                        xr[N3 - j] = make_float2(u.x - v.x, u.y - v.y);
                        a0.x += xr[j].x;
                        a0.y += xr[j].y;
                    }
                    const float2 mid = (N3 % 2 == 0) ? xr[N3 / 2] : make_float2(0.f, 0.f);
                    float2 *out = a1 + j2 * c3 + sym3;  // m3 = m sits at index sym3 + m
                    out[0] = make_float2(a0.x + mid.x, a0.y + mid.y);
                    for (int m = 1; m <= sym3; ++m) {
                        const float2 *w = tw3m + (sym3 + m) * N3;  // e(m j / n3), j = 0..n3-1: broadcast
                        const float sg = (m & 1) ? -1.f : 1.f;
                        float2 A = make_float2(fmaf(sg, mid.x, xr[0].x), fmaf(sg, mid.y, xr[0].y));
                        float2 B = make_float2(0.f, 0.f);
#pragma unroll
                        for (int j = 1; j <= H; ++j) {
                            const float2 cs = w[j];
                            A.x = fmaf(xr[j].x, cs.x, A.x);
                            A.y = fmaf(xr[j].y, cs.x, A.y);
                            B.x = fmaf(xr[N3 - j].x, cs.y, B.x);
                            B.y = fmaf(xr[N3 - j].y, cs.y, B.y);
                        }
                        out[m] = make_float2(A.x - B.y, A.y + B.x);   // A + i B
                        out[-m] = make_float2(A.x + B.y, A.y - B.x);  // A - i B
                    }
                } else {
                    for (int i3 = 0; i3 < c3; ++i3) {
                        const float2 *w = tw3m + i3 * N3;  // the same row for every lane: broadcast reads
                        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                        for (int j3 = 0; j3 < N3; ++j3)
                            cmac(acc, xr[j3], w[j3]);
                        a1[j2 * c3 + i3] = acc;
                    }
                }
            }
        } else {
            for (int o = lane; o < n2 * c3; o += 32) {
                const int j2 = o / c3, i3 = o - j2 * c3, step = m3[i3];
                const float2 *x = xp + j2 * ld3;
                float2 acc = make_float2(0.f, 0.f);
                int idx = 0;
                for (int j3 = 0; j3 < n3; ++j3) {
                    cmac(acc, x[j3], tw3[idx]);
                    idx += step;
                    if (idx >= n3)
                        idx -= n3;
                }
                a1[o] = acc;
            }
        }
        __syncwarp();
        // stage 2: y2[d] = sum_j2 a1[j2][i3(d)] e(m2(d) j2 / n2)
        float2 *dst = Y2 + (row * n1 + j1) * cd;
        if (np2 > 0) {
            // a1[j2] <- a1[j2] + a1[n2 - j2], a1[n2 - j2] <- a1[j2] - a1[n2 - j2] for 0 < j2 < n2 / 2
            for (int t = lane; t < h2 * c3; t += 32) {
                const int j2 = 1 + t / c3, i3 = t - (j2 - 1) * c3;
                const float2 u = a1[j2 * c3 + i3], v = a1[(n2 - j2) * c3 + i3];
                a1[j2 * c3 + i3] = make_float2(u.x + v.x, u.y + v.y);
                a1[(n2 - j2) * c3 + i3] = make_float2(u.x - v.x, u.y - v.y);
            }
            __syncwarp();
            for (int e = lane; e < np2; e += 32) {
                const int4 pr = pair2[e];  // (i3, m2, d of m2, d of -m2)
                const float2 *a = a1 + pr.x, *w = tw2m + pr.y * ld2;
                float2 A = a[0], B = make_float2(0.f, 0.f);
                if ((n2 & 1) == 0) {
                    const float sg = (pr.y & 1) ? -1.f : 1.f;
                    A.x = fmaf(sg, a[(n2 / 2) * c3].x, A.x);
                    A.y = fmaf(sg, a[(n2 / 2) * c3].y, A.y);
                }
                for (int j2 = 1; j2 <= h2; ++j2) {
                    const float2 cs = w[j2], s = a[j2 * c3], t = a[(n2 - j2) * c3];
                    A.x = fmaf(s.x, cs.x, A.x);
                    A.y = fmaf(s.y, cs.x, A.y);
                    B.x = fmaf(t.x, cs.y, B.x);
                    B.y = fmaf(t.y, cs.y, B.y);
                }
                dst[pr.z] = make_float2(A.x - B.y, A.y + B.x);      // A + i B
                if (pr.w >= 0)
                    dst[pr.w] = make_float2(A.x + B.y, A.y - B.x);  // A - i B
            }
        } else {
            for (int d = lane; d < cd; d += 32) {
                const int i3 = disk[2 * d + 1];
                const float2 *w = tw2d + d * (n2 + 1), *a = a1 + i3;
                float2 acc = make_float2(0.f, 0.f);
                for (int j2 = 0; j2 < n2; ++j2)
                    cmac(acc, a[j2 * c3], w[j2]);
                dst[d] = acc;
            }
        }
        __syncwarp();  // the plane buffer is rewritten by the next task
    }
}

// ---------------------------------------------------------------------------------------------
// Stages 1 and 2 with constant twiddles: square planes (n2 = n3 = N, a compiled size), spheres
// whose m3 values are exactly -M..M and whose disk is symmetric in m2.  The sums are the paired
// sums above, but every cos(2 pi m j / N) and sin(2 pi m j / N) is a compile-time constant, so
// each FMA takes its twiddle as an immediate operand and neither stage reads a table.  Stage 1
// keeps one line j2 per lane (outputs m3 = -M..M) and writes them transposed, a1t[i3][j2];
// stage 2 keeps one column i3 per lane and makes the outputs (+-m2, m3) for m2 = 0..k2.  The
// shared-memory traffic per plane is the staged plane, the transposed a1 and the cd outputs,
// against one broadcast twiddle read per four FMAs in the table form.
//
// The constants (twiddle_const.cuh) are the Taylor series of cosine and sine after an exact integer
// reduction of the angle to [0, pi/4], evaluated in FP64 by the compiler and rounded to FP32 once
// (the same values as the FP64-derived tables of the other kernels, up to the last bit of FP64).
using twiddle::kcos;
using twiddle::ksin;

// One term j of the paired sums of output m: A += s_j cos, B += t_j sin (s_j in x[j], t_j in
// x[N - j]); a zero constant drops its FMAs.
template <int N, int M, int J>
__device__ __forceinline__ void pterm(const float2 (&x)[N], float2 &A, float2 &B)
{
    constexpr float c = kcos<N, M * J>, s = ksin<N, M * J>;
    if constexpr (c != 0.f) {
        A.x = fmaf(x[J].x, c, A.x);
        A.y = fmaf(x[J].y, c, A.y);
    }
    if constexpr (s != 0.f) {
        B.x = fmaf(x[N - J].x, s, B.x);
        B.y = fmaf(x[N - J].y, s, B.y);
    }
}

// A = x_0 + (-1)^M x_{N/2} + sum_{0<j<N/2} s_j cos(2 pi M j / N),  B = sum_{0<j<N/2} t_j sin(2 pi M j / N)
template <int N, int M, int... J>
__device__ __forceinline__ void paired_sums(const float2 (&x)[N], float2 &A, float2 &B,
                                            std::integer_sequence<int, J...>)
{
    A = x[0];
    if constexpr (N % 2 == 0) {
        constexpr float sg = (M & 1) ? -1.f : 1.f;
        A.x = fmaf(sg, x[N / 2].x, A.x);
        A.y = fmaf(sg, x[N / 2].y, A.y);
    }
    B = make_float2(0.f, 0.f);
    (pterm<N, M, J + 1>(x, A, B), ...);
}

// x[j] <- x[j] + x[N - j], x[N - j] <- x[j] - x[N - j] for 0 < j < N / 2
template <int N>
__device__ __forceinline__ void pair_fold(float2 (&x)[N])
{
#pragma unroll
    for (int j = 1; j <= (N - 1) / 2; ++j) {
        const float2 u = x[j], v = x[N - j];
        x[j] = make_float2(u.x + v.x, u.y + v.y);
        x[N - j] = make_float2(u.x - v.x, u.y - v.y);
    }
}

// Stage-1 outputs m3 = +-Mo of a line (Mo <= M at run time): a1t rows M + Mo and M - Mo.  With
// sgn = -1 (negative exponent) the sine sums change sign.
template <int N, int Mo>
__device__ __forceinline__ void stage1_out(const float2 (&x)[N], int M, float sgn, float2 *col, int lda)
{
    if (Mo <= M) {
        float2 A, B;
        paired_sums<N, Mo>(x, A, B, std::make_integer_sequence<int, (N - 1) / 2>{});
        const float bx = sgn * B.x, by = sgn * B.y;
        col[(M + Mo) * lda] = make_float2(A.x - by, A.y + bx);
        col[(M - Mo) * lda] = make_float2(A.x + by, A.y - bx);
    }
}

// Stage-2 outputs (+-Mo, m3) of a column (Mo <= k2 at run time), into ys at the disk indices
// dt[Mo] = (index of +Mo, index of -Mo or -1).
template <int N, int Mo>
__device__ __forceinline__ void stage2_out(const float2 (&y)[N], int k2, float sgn, const int2 *dt, float2 *ys)
{
    if (Mo <= k2) {
        float2 A, B;
        paired_sums<N, Mo>(y, A, B, std::make_integer_sequence<int, (N - 1) / 2>{});
        const int2 d = dt[Mo];
        const float bx = sgn * B.x, by = sgn * B.y;
        if (d.x >= 0)
            ys[d.x] = make_float2(A.x - by, A.y + bx);
        if (Mo > 0 && d.y >= 0)
            ys[d.y] = make_float2(A.x + by, A.y - bx);
    }
}

// Two outputs Ma, Mb in one block: their eight accumulator chains interleave (four per output
// would leave each FMA waiting on the previous one of its chain).  Every accumulator still takes
// its terms in the order of paired_sums, so the results are the same bit for bit.
template <int N, int Ma, int Mb, int J>
__device__ __forceinline__ void pterm2(const float2 (&x)[N], float2 &A, float2 &B, float2 &C, float2 &D)
{
    pterm<N, Ma, J>(x, A, B);
    pterm<N, Mb, J>(x, C, D);
}

template <int N, int Ma, int Mb, int... J>
__device__ __forceinline__ void paired_sums2(const float2 (&x)[N], float2 &A, float2 &B, float2 &C, float2 &D,
                                             std::integer_sequence<int, J...>)
{
    A = x[0];
    C = x[0];
    if constexpr (N % 2 == 0) {
        constexpr float sa = (Ma & 1) ? -1.f : 1.f, sb = (Mb & 1) ? -1.f : 1.f;
        A.x = fmaf(sa, x[N / 2].x, A.x);
        A.y = fmaf(sa, x[N / 2].y, A.y);
        C.x = fmaf(sb, x[N / 2].x, C.x);
        C.y = fmaf(sb, x[N / 2].y, C.y);
    }
    B = make_float2(0.f, 0.f);
    D = B;
    (pterm2<N, Ma, Mb, J + 1>(x, A, B, C, D), ...);
}

// Stage-1 outputs Mo and Mo + 1 together when both are wanted, else Mo alone (Mo odd).
template <int N, int Mo>
__device__ __forceinline__ void stage1_out2(const float2 (&x)[N], int M, float sgn, float2 *col, int lda)
{
    if constexpr (Mo + 1 <= (N - 1) / 2) {
        if (Mo + 1 <= M) {
            float2 A, B, C, D;
            paired_sums2<N, Mo, Mo + 1>(x, A, B, C, D, std::make_integer_sequence<int, (N - 1) / 2>{});
            const float bx = sgn * B.x, by = sgn * B.y, dx = sgn * D.x, dy = sgn * D.y;
            col[(M + Mo) * lda] = make_float2(A.x - by, A.y + bx);
            col[(M - Mo) * lda] = make_float2(A.x + by, A.y - bx);
            col[(M + Mo + 1) * lda] = make_float2(C.x - dy, C.y + dx);
            col[(M - Mo - 1) * lda] = make_float2(C.x + dy, C.y - dx);
            return;
        }
    }
    stage1_out<N, Mo>(x, M, sgn, col, lda);
}

template <int N, int... I>
__device__ __forceinline__ void stage1_all2(const float2 (&x)[N], int M, float sgn, float2 *col, int lda,
                                            std::integer_sequence<int, I...>)
{
    (stage1_out2<N, 2 * I + 1>(x, M, sgn, col, lda), ...);
}

// Stage-2 outputs Mo and Mo + 1 together when both are wanted, else Mo alone (Mo even).
template <int N, int Mo>
__device__ __forceinline__ void stage2_out2(const float2 (&y)[N], int k2, float sgn, const int2 *dt, float2 *ys)
{
    if constexpr (Mo + 1 <= (N - 1) / 2) {
        if (Mo + 1 <= k2) {
            float2 A, B, C, D;
            paired_sums2<N, Mo, Mo + 1>(y, A, B, C, D, std::make_integer_sequence<int, (N - 1) / 2>{});
            const int2 da = dt[Mo], db = dt[Mo + 1];
            const float bx = sgn * B.x, by = sgn * B.y, dx = sgn * D.x, dy = sgn * D.y;
            if (da.x >= 0)
                ys[da.x] = make_float2(A.x - by, A.y + bx);
            if (Mo > 0 && da.y >= 0)
                ys[da.y] = make_float2(A.x + by, A.y - bx);
            if (db.x >= 0)
                ys[db.x] = make_float2(C.x - dy, C.y + dx);
            if (db.y >= 0)
                ys[db.y] = make_float2(C.x + dy, C.y - dx);
            return;
        }
    }
    stage2_out<N, Mo>(y, k2, sgn, dt, ys);
}

template <int N, int... I>
__device__ __forceinline__ void stage2_all2(const float2 (&y)[N], int k2, float sgn, const int2 *dt, float2 *ys,
                                            std::integer_sequence<int, I...>)
{
    (stage2_out2<N, 2 * I>(y, k2, sgn, dt, ys), ...);
}

// Per warp: the staged plane [N][p12_pitch(N)] (two of them in the asynchronous form), then a1t
// [c3][N | 1] of two planes (an odd pitch: lanes on different columns read different banks), each
// reused for that plane's cd outputs; an even count of float2 so the next warp's plane stays
// 16-byte aligned.
constexpr int P12A_WARPS = 7;  // the asynchronous form: two CTAs of 7 warps fit an SM's shared memory

__host__ __device__ inline size_t p12c_warp_floats2(int N, int c3, bool async = false)
{
    return ((async ? 2 : 1) * (size_t)N * p12_pitch(N) + 2 * (size_t)c3 * (N | 1) + 1) & ~(size_t)1;
}

__host__ __device__ inline size_t p12c_smem(int N, int c3, bool async = false)
{
    return align16(sizeof(int2) * (size_t)c3 * ((N - 1) / 2 + 1)) +
           (async ? P12A_WARPS : P12_WARPS) * p12c_warp_floats2(N, c3, async) * sizeof(float2);
}

constexpr int P12C_MAX_C3 = 16;  // stage 2 runs two planes side by side, one per half-warp

// A warp takes two tasks (planes) at a time: stage 1 of each (a lane per line), then stage 2 of
// both together, lanes 0-15 on the first plane's columns and lanes 16-31 on the second's, so a
// sphere with c3 <= 16 keeps twice as many lanes busy in stage 2 as one plane would.
//
// ASYNC (plain rows, even N, 16-byte aligned rows): the planes arrive by cp.async into two buffers
// per warp, the next pair's first plane issued once this pair's first plane has been read and its
// second plane once the second has been read, so the copies run behind the other plane's stage 1
// and stage 2 instead of stalling the warp; 7 warps per CTA keep two CTAs per SM.
template <int N, bool PAIR, bool ASYNC = false>  // two CTAs per SM (shared memory allows two at every compiled N)
__global__ void __launch_bounds__((ASYNC ? P12A_WARPS : P12_WARPS) * 32, 2)
    dft_plane12c_kernel(const float2 *__restrict__ X, long long ldx, int rows, int n1, int M, int cd, int np2, int k2,
                        const int4 *__restrict__ g_pair2, float sgn, float2 *__restrict__ Y2, PairSrc ps)
{
    static_assert(!ASYNC || (!PAIR && N % 2 == 0), "the asynchronous form takes plain rows of even N");
    constexpr int NWARPS = ASYNC ? P12A_WARPS : P12_WARPS;
    constexpr int H = (N - 1) / 2;
    constexpr int SP = p12_pitch(N);
    constexpr int LDA = N | 1;
    constexpr int plane = N * N;
    extern __shared__ __align__(16) uint8_t smem[];
    const int c3 = 2 * M + 1;
    int2 *dtab = reinterpret_cast<int2 *>(smem);  // [c3][H + 1]
    float2 *wbase = reinterpret_cast<float2 *>(smem + align16(sizeof(int2) * (size_t)c3 * (H + 1)));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int t = tid; t < c3 * (H + 1); t += blockDim.x)
        dtab[t] = make_int2(-1, -1);
    __syncthreads();
    for (int t = tid; t < np2; t += blockDim.x) {
        const int4 pr = g_pair2[t];  // (i3, m2 >= 0, disk index of m2, of -m2 or -1)
        dtab[pr.x * (H + 1) + pr.y] = make_int2(pr.z, pr.w);
    }
    __syncthreads();
    float2 *pl = wbase + (size_t)warp * p12c_warp_floats2(N, c3, ASYNC);  // [N][SP]
    float2 *pl2 = pl + (ASYNC ? N * SP : 0);                               // ASYNC: the second buffer
    float2 *a1t0 = pl2 + N * SP;                                           // [c3][LDA], first plane
    float2 *a1t1 = a1t0 + c3 * LDA;                                        // [c3][LDA], second plane
    const bool vec = (N % 2 == 0) && (ldx % 2 == 0) && ((reinterpret_cast<size_t>(X) & 15) == 0);
    // task -> (row, j1): plain rows row-major, pair rows j1-major (the warps of a CTA share psi_v);
    // 32-bit arithmetic (the launcher keeps rows n1 below 2^31)
    const unsigned ntasks = (unsigned)rows * (unsigned)n1, npairs = (ntasks + 1) / 2;
    auto locate = [&](unsigned task, long long &row, int &j1) {
        if (PAIR) {
            const unsigned q = task / (unsigned)rows;
            j1 = (int)q;
            row = (long long)(task - q * (unsigned)rows);
        } else {
            const unsigned q = task / (unsigned)n1;
            row = (long long)q;
            j1 = (int)(task - q * (unsigned)n1);
        }
    };
    // one plane into pl (pair densities formed on the way)
    auto load_plane = [&](long long row, int j1) {
        const float2 *src, *srcv = nullptr;
        float w = 0.f;
        if (PAIR) {
            const int kk = (int)row, v = kk / ps.nc;
            src = X + (size_t)(ps.c0 + kk - v * ps.nc) * ldx + (size_t)j1 * plane;
            srcv = X + (size_t)v * ldx + (size_t)j1 * plane;
            w = ps.sw[kk];
        } else {
            src = X + row * ldx + (size_t)j1 * plane;
        }
        if (N % 2 == 0 && vec) {
            constexpr int QR = N / 2;  // 16-byte words per line
            const float4 *s4 = reinterpret_cast<const float4 *>(src);
            const float4 *v4 = reinterpret_cast<const float4 *>(srcv);
            constexpr int UNR = PAIR ? 4 : 8;  // loads in flight per lane (pair rows load two values)
#pragma unroll UNR
            for (int q = lane; q < N * QR; q += 32) {
                const int j2 = q / QR, c = q - j2 * QR;
                float4 x = __ldg(s4 + q);
                if (PAIR) {
                    const float4 a = __ldg(v4 + q);
                    const float2 lo = pair_or_x<PAIR>(make_float2(a.x, a.y), make_float2(x.x, x.y), w);
                    const float2 hi = pair_or_x<PAIR>(make_float2(a.z, a.w), make_float2(x.z, x.w), w);
                    x = make_float4(lo.x, lo.y, hi.x, hi.y);
                }
                *reinterpret_cast<float4 *>(pl + j2 * SP + 2 * c) = x;
            }
        } else {
#pragma unroll 8
            for (int q = lane; q < plane; q += 32) {
                const int j2 = q / N, j3 = q - j2 * N;
                const float2 xs = __ldg(src + q);
                pl[j2 * SP + j3] = PAIR ? pair_or_x<true>(__ldg(srcv + q), xs, w) : xs;
            }
        }
        __syncwarp();
    };
    // stage 1 of the plane in buffer b: a1t[M + m3][j2] = sum_j3 x[j2][j3] e(+-m3 j3 / N)
    auto stage1 = [&](const float2 *b, float2 *a1t) {
        for (int j2 = lane; j2 < N; j2 += 32) {
            float2 x[N];
            const float2 *ls = b + j2 * SP;
            if constexpr (N % 2 == 0) {
#pragma unroll
                for (int j = 0; j < N; j += 2) {
                    const float4 v = *reinterpret_cast<const float4 *>(ls + j);
                    x[j] = make_float2(v.x, v.y);
                    x[j + 1] = make_float2(v.z, v.w);
                }
            } else {
#pragma unroll
                for (int j = 0; j < N; ++j)
                    x[j] = ls[j];
            }
            pair_fold<N>(x);
            float2 a0 = x[0];
#pragma unroll
            for (int j = 1; j <= H; ++j) {  // the m3 = 0 sum, in the order of the table form
                a0.x += x[j].x;
                a0.y += x[j].y;
            }
            float2 *col = a1t + j2;
            if constexpr (N % 2 == 0)
                col[M * LDA] = make_float2(a0.x + x[N / 2].x, a0.y + x[N / 2].y);
            else
                col[M * LDA] = a0;
            stage1_all2<N>(x, M, sgn, col, LDA, std::make_integer_sequence<int, (H + 1) / 2>{});
        }
        __syncwarp();  // the buffer is rewritten by a later plane
    };
    // stage 2 of a pair: ys[d] = sum_j2 a1t[i3][j2] e(+-m2 j2 / N) for the disk points
    // d = (m2, m3(i3)), written over the plane's a1t once every lane holds its column; then both
    // planes' cd values to the workspace
    auto stage2 = [&](long long rowA, int j1A, long long rowB, int j1B, bool hasB) {
        const int half = lane >> 4, i3 = lane & 15;
        float2 *a1t = half ? a1t1 : a1t0;
        const bool act = i3 < c3 && (half == 0 || hasB);
        float2 y[N];
        if (act) {
            const float2 *cs = a1t + i3 * LDA;
#pragma unroll
            for (int j = 0; j < N; ++j)
                y[j] = cs[j];
        }
        __syncwarp();
        if (act) {
            pair_fold<N>(y);
            stage2_all2<N>(y, k2, sgn, dtab + i3 * (H + 1), a1t, std::make_integer_sequence<int, H / 2 + 1>{});
        }
        __syncwarp();
        float2 *dA = Y2 + (rowA * n1 + j1A) * cd;
        for (int t = lane; t < cd; t += 32)
            dA[t] = a1t0[t];
        if (hasB) {
            float2 *dB = Y2 + (rowB * n1 + j1B) * cd;
            for (int t = lane; t < cd; t += 32)
                dB[t] = a1t1[t];
        }
        __syncwarp();  // a1t is rewritten by the next pair
    };
    const unsigned ustride = gridDim.x * NWARPS;
    if constexpr (ASYNC) {
        // the plane of task t into buffer b with 16-byte cp.async, one group (an empty group when
        // t is past the end, so that every wait below sees the same count of groups)
        auto issue = [&](unsigned t, float2 *b) {
            if (t < ntasks) {
                long long row;
                int j1;
                locate(t, row, j1);
                const float2 *src = X + row * ldx + (size_t)j1 * plane;
                constexpr int QR = N / 2;
#pragma unroll 4
                for (int q = lane; q < N * QR; q += 32) {
                    const int j2 = q / QR, c = q - j2 * QR;
                    cp_async16(b + j2 * SP + 2 * c, src + 2 * q);
                }
            }
            cp_async_commit();
        };
        unsigned u = blockIdx.x * NWARPS + warp;
        issue(2 * u, pl);
        issue(2 * u + 1, pl2);
        for (; u < npairs; u += ustride) {
            const unsigned tA = 2 * u, tB = tA + 1, nA = 2 * (u + ustride);
            const bool hasB = tB < ntasks;
            long long rowA, rowB = 0;
            int j1A, j1B = 0;
            locate(tA, rowA, j1A);
            if (hasB)
                locate(tB, rowB, j1B);
            cp_async_wait<1>();  // groups in flight: this pair's A and B; A is in
            __syncwarp();
            stage1(pl, a1t0);
            issue(nA < 2 * npairs ? nA : ntasks, pl);  // the next pair's A (or an empty group)
            cp_async_wait<1>();                        // B is in
            __syncwarp();
            if (hasB)
                stage1(pl2, a1t1);
            issue(nA + 1 < 2 * npairs ? nA + 1 : ntasks, pl2);  // the next pair's B
            stage2(rowA, j1A, rowB, j1B, hasB);
        }
        cp_async_wait<0>();
    } else {
        for (unsigned u = blockIdx.x * NWARPS + warp; u < npairs; u += ustride) {
            const unsigned tA = 2 * u, tB = tA + 1;
            const bool hasB = tB < ntasks;
            long long rowA, rowB = 0;
            int j1A, j1B = 0;
            locate(tA, rowA, j1A);
            load_plane(rowA, j1A);
            stage1(pl, a1t0);
            if (hasB) {
                locate(tB, rowB, j1B);
                load_plane(rowB, j1B);
                stage1(pl, a1t1);
            }
            stage2(rowA, j1A, rowB, j1B, hasB);
        }
    }
}

// Stage 3 with sphere pairs (np1 > 0): y(+-m1, d) = A +- i B from the sums of
// ys[j1][d] + ys[n1 - j1][d] (times the cosine) and ys[j1][d] - ys[n1 - j1][d] (times the sine),
// formed while the row is loaded; tw1m[m1][j1] = e(m1 j1 / n1), m1 <= k1, rows of p3_ld1 (odd).
__host__ __device__ inline int p3_ld1(int n1) { return (n1 / 2 + 1) | 1; }

__host__ __device__ inline size_t p3_smem_paired(int n1, int cd, int np1, int k1, int ng)
{
    return sizeof(int4) * np1 + align16(sizeof(float2) * (size_t)(k1 + 1) * p3_ld1(n1)) +
           2 * align16(sizeof(float2) * (size_t)n1 * cd) + sizeof(float2) * (size_t)ng;
}

// One CTA per row at a time, the rows double-buffered: the next row's n1 x cd values are copied
// into the second buffer with cp.async while this row's outputs are formed, so the workspace
// latency overlaps the arithmetic.  Then the pairs over j1 are formed in place and each thread
// makes the outputs of its sphere pairs, into shared memory (sphere order scatters them), from
// where the row is written with coalesced stores.
__global__ void __launch_bounds__(256)
    dft_stage3_paired_kernel(const float2 *__restrict__ Y2, int rows, int n1, int cd, int np1, int k1, int ng,
                             const int4 *__restrict__ g_pair1, const float2 *__restrict__ g_tw,
                             float2 *__restrict__ Y, long long ldy)
{
    extern __shared__ __align__(16) uint8_t smem[];
    int4 *pair1 = reinterpret_cast<int4 *>(smem);                // [np1]
    float2 *tw1m = reinterpret_cast<float2 *>(pair1 + np1);     // [k1 + 1][ld1]
    const int ld1 = p3_ld1(n1), h1 = (n1 - 1) / 2;
    const size_t rowv = (size_t)n1 * cd;
    float2 *buf0 = reinterpret_cast<float2 *>(reinterpret_cast<uint8_t *>(tw1m) +
                                              align16(sizeof(float2) * (size_t)(k1 + 1) * ld1));
    float2 *buf1 = reinterpret_cast<float2 *>(reinterpret_cast<uint8_t *>(buf0) + align16(sizeof(float2) * rowv));
    float2 *yo = reinterpret_cast<float2 *>(reinterpret_cast<uint8_t *>(buf1) + align16(sizeof(float2) * rowv));
    const int tid = threadIdx.x;
    for (int t = tid; t < np1; t += blockDim.x)
        pair1[t] = g_pair1[t];
    for (int t = tid; t < (k1 + 1) * ld1; t += blockDim.x) {
        const int m1 = t / ld1, j1 = t - m1 * ld1;
        tw1m[t] = g_tw[(m1 * j1) % n1];
    }
    // a row block is rowv values at Y2 + row rowv: 16-byte copies when every block starts on 16 bytes
    const bool v16 = (rowv % 2 == 0) && ((reinterpret_cast<size_t>(Y2) & 15) == 0);
    auto fetch = [&](long long row, float2 *dst) {
        const float2 *src = Y2 + row * (long long)rowv;
        if (v16) {
            for (int t = tid; t < (int)(rowv / 2); t += blockDim.x)
                cp_async16(dst + 2 * t, src + 2 * t);
        } else {
            for (int t = tid; t < (int)rowv; t += blockDim.x)
                cp_async8(dst + t, src + t);
        }
        cp_async_commit();
    };
    long long row = blockIdx.x;
    if (row < rows)
        fetch(row, buf0);
    for (int it = 0; row < rows; ++it, row += gridDim.x) {
        float2 *ys = (it & 1) ? buf1 : buf0;
        const long long next = row + gridDim.x;
        if (next < rows)
            fetch(next, (it & 1) ? buf0 : buf1);  // its buffer was last read before the previous row's final barrier
        else
            cp_async_commit();  // an empty group keeps the count of groups in flight at two
        cp_async_wait<1>();     // this thread's copies of the current row are done
        __syncthreads();        // everyone's are (and the tables are ready on the first row)
        for (int t = tid; t < h1 * cd; t += blockDim.x) {
            const int j1 = 1 + t / cd, d = t - (j1 - 1) * cd;
            const float2 u = ys[j1 * cd + d], v = ys[(n1 - j1) * cd + d];
            ys[j1 * cd + d] = make_float2(u.x + v.x, u.y + v.y);
            ys[(n1 - j1) * cd + d] = make_float2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
        for (int e = tid; e < np1; e += blockDim.x) {
            const int4 pr = pair1[e];  // (d, m1, g of m1, g of -m1)
            const float2 *a = ys + pr.x, *w = tw1m + pr.y * ld1;
            float2 A = a[0], B = make_float2(0.f, 0.f);
            if ((n1 & 1) == 0) {
                const float sg = (pr.y & 1) ? -1.f : 1.f;
                A.x = fmaf(sg, a[(n1 / 2) * cd].x, A.x);
                A.y = fmaf(sg, a[(n1 / 2) * cd].y, A.y);
            }
            for (int j1 = 1; j1 <= h1; ++j1) {
                const float2 cs = w[j1], s = a[j1 * cd], t = a[(n1 - j1) * cd];
                A.x = fmaf(s.x, cs.x, A.x);
                A.y = fmaf(s.y, cs.x, A.y);
                B.x = fmaf(t.x, cs.y, B.x);
                B.y = fmaf(t.y, cs.y, B.y);
            }
            yo[pr.z] = make_float2(A.x - B.y, A.y + B.x);      // A + i B
            if (pr.w >= 0)
                yo[pr.w] = make_float2(A.x + B.y, A.y - B.x);  // A - i B
        }
        __syncthreads();  // yo is complete, and ys is free to be refilled two rows on
        float2 *y = Y + row * ldy;
        for (int g = tid; g < ng; g += blockDim.x)
            y[g] = yo[g];
    }
    cp_async_wait<0>();
}

// Stage 3 with constant twiddles (n1 a compiled size up to 27, sphere pairs present): a thread per
// disk point d.  It reads its n1 values ys[j1][d] (consecutive threads on consecutive d, so no
// bank conflicts), forms the pairs over j1 in registers and makes the outputs (+-m1, d) for
// m1 = 0..k1 with the twiddles as compile-time constants (the same sums, in the same order, as
// dft_stage3_paired_kernel); entries of the sphere table gtab[d][m1] that are -1 are skipped.
// Each CTA takes R rows at a time (R cdp threads, cdp = cd rounded up to 32), double-buffered by
// cp.async; the outputs go through shared memory to coalesced stores.
__host__ __device__ inline int p3c_cdp(int cd) { return (cd + 31) & ~31; }
__host__ __device__ inline int p3c_rows(int cd) { return p3c_cdp(cd) >= 256 ? 1 : 256 / p3c_cdp(cd); }

__host__ __device__ inline size_t p3c_smem(int n1, int cd, int k1, int ng)
{
    const int R = p3c_rows(cd);
    return align16(sizeof(int2) * (size_t)cd * (k1 + 1)) + 2 * align16(sizeof(float2) * (size_t)R * n1 * cd) +
           sizeof(float2) * (size_t)R * ng;
}

template <int N1>
__global__ void __launch_bounds__(256)
    dft_stage3c_kernel(const float2 *__restrict__ Y2, int rows, int cd, int np1, int k1, int ng,
                       const int4 *__restrict__ g_pair1, float sgn, float2 *__restrict__ Y, long long ldy)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int R = p3c_rows(cd), cdp = p3c_cdp(cd);
    const size_t rowv = (size_t)N1 * cd;
    int2 *gtab = reinterpret_cast<int2 *>(smem);  // [cd][k1 + 1]: sphere index of (+m1, d), of (-m1, d)
    float2 *buf0 = reinterpret_cast<float2 *>(smem + align16(sizeof(int2) * (size_t)cd * (k1 + 1)));
    float2 *buf1 = reinterpret_cast<float2 *>(reinterpret_cast<uint8_t *>(buf0) + align16(sizeof(float2) * R * rowv));
    float2 *yo = reinterpret_cast<float2 *>(reinterpret_cast<uint8_t *>(buf1) + align16(sizeof(float2) * R * rowv));
    const int tid = threadIdx.x;
    for (int t = tid; t < cd * (k1 + 1); t += blockDim.x)
        gtab[t] = make_int2(-1, -1);
    __syncthreads();
    for (int t = tid; t < np1; t += blockDim.x) {
        const int4 pr = g_pair1[t];  // (d, m1 >= 0, g of m1, g of -m1 or -1)
        gtab[pr.x * (k1 + 1) + pr.y] = make_int2(pr.z, pr.w);
    }
    const int rl = tid / cdp, d = tid - rl * cdp;
    const bool v16 = (rowv % 2 == 0) && ((reinterpret_cast<size_t>(Y2) & 15) == 0);
    // rows [r0, r0 + R) are contiguous in the workspace
    auto fetch = [&](long long r0, float2 *dst) {
        const float2 *src = Y2 + r0 * (long long)rowv;
        const long long nv = (long long)min((long long)R, rows - r0) * (long long)rowv;
        if (v16) {
            for (long long t = tid; t < nv / 2; t += blockDim.x)
                cp_async16(dst + 2 * t, src + 2 * t);
        } else {
            for (long long t = tid; t < nv; t += blockDim.x)
                cp_async8(dst + t, src + t);
        }
        cp_async_commit();
    };
    long long r0 = (long long)blockIdx.x * R;
    const long long rstride = (long long)gridDim.x * R;
    if (r0 < rows)
        fetch(r0, buf0);
    for (int it = 0; r0 < rows; ++it, r0 += rstride) {
        float2 *ys = (it & 1) ? buf1 : buf0;
        if (r0 + rstride < rows)
            fetch(r0 + rstride, (it & 1) ? buf0 : buf1);  // read last before the previous group's barrier
        else
            cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const int nr = (int)min((long long)R, rows - r0);
        if (rl < nr && d < cd) {
            float2 x[N1];
            const float2 *c = ys + rl * rowv + d;
#pragma unroll
            for (int j = 0; j < N1; ++j)
                x[j] = c[j * cd];
            pair_fold<N1>(x);
            stage2_all2<N1>(x, k1, sgn, gtab + d * (k1 + 1), yo + rl * ng,
                            std::make_integer_sequence<int, (N1 - 1) / 2 / 2 + 1>{});
        }
        __syncthreads();  // yo is complete, and ys is free to be refilled
        for (int t = tid; t < nr * ng; t += blockDim.x) {
            const int r = t / ng, g = t - r * ng;
            Y[(r0 + r) * ldy + g] = yo[t];
        }
    }
    cp_async_wait<0>();
}

__global__ void __launch_bounds__(256)
    dft_stage3_kernel(const float2 *__restrict__ Y2, int rows, int n1, int cd, int ng, const int *__restrict__ g_gmap,
                      const float2 *__restrict__ g_tw, float2 *__restrict__ Y, long long ldy)
{
    extern __shared__ __align__(16) uint8_t smem[];
    float2 *ys = reinterpret_cast<float2 *>(smem);      // [n1][cd]
    float2 *tw1 = ys + (size_t)n1 * cd;                 // [n1]
    int *gmap = reinterpret_cast<int *>(tw1 + n1);      // [ng][2]
    const int tid = threadIdx.x;
    for (int t = tid; t < n1; t += blockDim.x)
        tw1[t] = g_tw[t];
    for (int t = tid; t < 2 * ng; t += blockDim.x)
        gmap[t] = g_gmap[t];
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        __syncthreads();  // tables ready / previous row's reads done
        const float2 *src = Y2 + row * n1 * cd;
        for (int t = tid; t < n1 * cd; t += blockDim.x)
            ys[t] = src[t];
        __syncthreads();
        for (int g = tid; g < ng; g += blockDim.x) {
            const int step = gmap[2 * g], d = gmap[2 * g + 1];
            float2 acc = make_float2(0.f, 0.f);
            int idx = 0;
            for (int j1 = 0; j1 < n1; ++j1) {
                cmac(acc, ys[j1 * cd + d], tw1[idx]);
                idx += step;
                if (idx >= n1)
                    idx -= n1;
            }
            Y[row * ldy + g] = acc;
        }
    }
}

constexpr size_t DFT_SMEM_TARGET = 56 * 1024;  // four CTAs per SM
constexpr size_t DFT_SMEM_MAX = 220 * 1024;

int rows_per_cta(const DftPlan &p)
{
    for (int R : {4, 2})
        if (layout_for(p.n, p.ng, p.c3, p.cd, R).total <= DFT_SMEM_TARGET && R * p.ng <= DFT_THREADS * GPT_MAX)
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

bool dft_supported(const DftPlan &p)
{
    return p.ng <= DFT_THREADS * GPT_MAX && layout_for(p.n, p.ng, p.c3, p.cd, 1).total <= DFT_SMEM_MAX;
}

template <int R, int GPT>
static cudaError_t launch_dft_RG(const float2 *X, long long ldx, int rows, float2 *Y, long long ldy, const DftPlan &p,
                                 cudaStream_t s, const float2 *tw)
{
    const size_t smem = layout_for(p.n, p.ng, p.c3, p.cd, R).total;
    cudaError_t e =
        cudaFuncSetAttribute(dft_rows_kernel<R, GPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    dft_rows_kernel<R, GPT><<<(rows + R - 1) / R, DFT_THREADS, smem, s>>>(
        X, ldx, rows, Y, ldy, p.n[0], p.n[1], p.n[2], p.ng, p.c3, p.cd, p.m3list, p.disk, p.gmap, tw);
    count_launches(1);
    return cudaGetLastError();
}

template <int R>
static cudaError_t launch_dft_R(const float2 *X, long long ldx, int rows, float2 *Y, long long ldy, const DftPlan &p,
                                cudaStream_t s, const float2 *tw)
{
    const int need = (R * p.ng + DFT_THREADS - 1) / DFT_THREADS;  // stage-3 outputs per thread
    if (need <= 4)
        return launch_dft_RG<R, 4>(X, ldx, rows, Y, ldy, p, s, tw);
    if (need <= 8)
        return launch_dft_RG<R, 8>(X, ldx, rows, Y, ldy, p, s, tw);
    if (need <= 12)
        return launch_dft_RG<R, 12>(X, ldx, rows, Y, ldy, p, s, tw);
    return launch_dft_RG<R, 16>(X, ldx, rows, Y, ldy, p, s, tw);
}

// With the register stage 1 the plane-per-warp form is the faster one for every row count; its
// workspace holds n1 cd values per row.  Grids whose n3 has no compiled stage 1 keep the
// row-block kernel for long transforms (it reads 1.25 shared-memory words per complex FMA against
// two for the generic plane-per-warp stage 1).
constexpr int WS_MAX_ROWS_GENERIC = 4096;

bool p12_compiled(int n3)
{
    switch (n3) {
    case 12: case 16: case 18: case 20: case 24: case 27: case 30: case 32: case 36:
        return true;
    default:
        return false;
    }
}

size_t dft_work_bytes(const DftPlan &p, int rows)
{
    const int r = p12_compiled(p.n[2]) ? rows : std::min(rows, WS_MAX_ROWS_GENERIC);
    return (size_t)r * p.n[0] * p.cd * sizeof(float2);
}

template <int N3, bool PAIR>
static cudaError_t launch_p12_t(int grid, size_t smem, const float2 *X, long long ldx, int rows, const DftPlan &p,
                                const float2 *tw, float2 *work, PairSrc ps, cudaStream_t s)
{
    if (N3 > 0 && N3 % 2 == 0)  // the staged plane rows
        smem = p12_smem(p.n, p.c3, p.cd, p.np2, p.k2, false, true);
    if (smem > DFT_SMEM_MAX)
        return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(dft_plane12_kernel<N3, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    dft_plane12_kernel<N3, PAIR><<<grid, P12_WARPS * 32, smem, s>>>(X, ldx, rows, p.n[0], p.n[1], p.n[2], p.c3,
                                                                     p.sym3, p.cd, p.m3list, p.disk, p.np2, p.k2,
                                                                     p.pair2, tw, work, ps);
    return cudaGetLastError();
}

template <int N, bool PAIR, bool ASYNC>
static cudaError_t launch_p12c_t(int grid, const float2 *X, long long ldx, int rows, const DftPlan &p, float sgn,
                                 float2 *work, PairSrc ps, cudaStream_t s)
{
    const size_t smem = p12c_smem(N, p.c3, ASYNC);
    cudaError_t e = cudaFuncSetAttribute(dft_plane12c_kernel<N, PAIR, ASYNC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    dft_plane12c_kernel<N, PAIR, ASYNC><<<grid, (ASYNC ? P12A_WARPS : P12_WARPS) * 32, smem, s>>>(
        X, ldx, rows, p.n[0], p.sym3, p.cd, p.np2, p.k2, p.pair2, sgn, work, ps);
    return cudaGetLastError();
}

// Plain rows of even N on 16-byte boundaries take the asynchronous form.
template <int N>
static cudaError_t launch_p12c(int grid, const float2 *X, long long ldx, int rows, const DftPlan &p, float sgn,
                               float2 *work, const PairSrc *ps, cudaStream_t s)
{
    if (ps)
        return launch_p12c_t<N, true, false>(grid, X, ldx, rows, p, sgn, work, *ps, s);
    if constexpr (N % 2 == 0) {
        if (ldx % 2 == 0 && (reinterpret_cast<size_t>(X) & 15) == 0 &&
            p12c_smem(N, p.c3, true) <= DFT_SMEM_MAX) {
            const long long ntasks = (long long)rows * p.n[0];
            const int ga = (int)std::min<long long>((ntasks + P12A_WARPS - 1) / P12A_WARPS, 152LL * 16);
            return launch_p12c_t<N, false, true>(ga, X, ldx, rows, p, sgn, work, PairSrc{nullptr, 0, 1, 0}, s);
        }
    }
    return launch_p12c_t<N, false, false>(grid, X, ldx, rows, p, sgn, work, PairSrc{nullptr, 0, 1, 0}, s);
}

template <int N1>
static cudaError_t launch_p3c(int grid, int nthr, size_t smem, const float2 *work, int rows, const DftPlan &p, float sgn,
                              float2 *Y, long long ldy, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(dft_stage3c_kernel<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    dft_stage3c_kernel<N1><<<grid, nthr, smem, s>>>(work, rows, p.cd, p.np1, p.k1, p.ng, p.pair1, sgn, Y, ldy);
    return cudaGetLastError();
}

// The constant-twiddle stages 1 and 2 serve square planes with N <= 27 (larger lines would not fit
// two CTAs' registers per SM) and spheres whose m3 values are -M..M, M <= 7, with a disk symmetric
// in m2 (every sphere at q = 0).
static bool p12c_compiled(int N)
{
    return N == 12 || N == 16 || N == 18 || N == 20 || N == 24 || N == 27;
}

static bool p12c_applies(const DftPlan &p)
{
    const int N = p.n[2];
    return p.n[1] == N && p12c_compiled(N) && p.sym3 >= 0 && p.c3 == 2 * p.sym3 + 1 && p.np2 > 0 &&
           p.c3 <= P12C_MAX_C3 && p.k2 <= (N - 1) / 2 && p12c_smem(N, p.c3) <= DFT_SMEM_MAX;
}

template <int N3>
static cudaError_t launch_p12(int grid, size_t smem, const float2 *X, long long ldx, int rows, const DftPlan &p,
                              const float2 *tw, float2 *work, const PairSrc *ps, cudaStream_t s)
{
    return ps ? launch_p12_t<N3, true>(grid, smem, X, ldx, rows, p, tw, work, *ps, s)
              : launch_p12_t<N3, false>(grid, smem, X, ldx, rows, p, tw, work, PairSrc{nullptr, 0, 1, 0}, s);
}

// The two-kernel transform of `rows` rows: of X (ps == nullptr) or of the pair densities formed
// from the states X = psi [nb][ldx] (ps != nullptr).  Returns cudaErrorNotSupported, with nothing
// launched, when pair rows would need the row-block kernel.
static cudaError_t dft_two_kernel(const float2 *X, long long ldx, int rows, float2 *Y, long long ldy,
                                  const DftPlan &p, float2 *work, cudaStream_t s, bool negative_exponent,
                                  const PairSrc *ps, bool const_twiddles)
{
    if (rows <= 0)
        return cudaSuccess;
    if ((!p12_compiled(p.n[2]) && rows > WS_MAX_ROWS_GENERIC) || !work)
        return ps ? cudaErrorNotSupported : launch_dft_rows(X, ldx, rows, Y, ldy, p, s, negative_exponent);
    const float2 *tw = negative_exponent ? p.twc : p.tw;
    const size_t sm12 = p12_smem(p.n, p.c3, p.cd, p.np2, p.k2, !p12_compiled(p.n[2]));
    const bool paired3 = p.np1 > 0 && p3_smem_paired(p.n[0], p.cd, p.np1, p.k1, p.ng) <= DFT_SMEM_MAX;
    const size_t sm3 = paired3 ? p3_smem_paired(p.n[0], p.cd, p.np1, p.k1, p.ng)
                               : sizeof(float2) * ((size_t)p.n[0] * p.cd + p.n[0]) + sizeof(int) * 2 * p.ng;
    const bool cst = const_twiddles && p12c_applies(p) && (long long)rows * p.n[0] < (1LL << 31);
    if ((!cst && sm12 > DFT_SMEM_MAX) || sm3 > DFT_SMEM_MAX)
        return ps ? cudaErrorNotSupported : launch_dft_rows(X, ldx, rows, Y, ldy, p, s, negative_exponent);
    cudaError_t e = paired3 ? cudaFuncSetAttribute(dft_stage3_paired_kernel,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3)
                            : cudaFuncSetAttribute(dft_stage3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)sm3);
    if (e != cudaSuccess)
        return e;
    const long long ntasks = (long long)rows * p.n[0];
    const int g12 = (int)std::min<long long>((ntasks + P12_WARPS - 1) / P12_WARPS, 152LL * 16);
    const float sgn = negative_exponent ? -1.f : 1.f;
    if (cst) {
        switch (p.n[2]) {
        case 12: e = launch_p12c<12>(g12, X, ldx, rows, p, sgn, work, ps, s); break;
        case 16: e = launch_p12c<16>(g12, X, ldx, rows, p, sgn, work, ps, s); break;
        case 18: e = launch_p12c<18>(g12, X, ldx, rows, p, sgn, work, ps, s); break;
        case 20: e = launch_p12c<20>(g12, X, ldx, rows, p, sgn, work, ps, s); break;
        case 24: e = launch_p12c<24>(g12, X, ldx, rows, p, sgn, work, ps, s); break;
        case 27: e = launch_p12c<27>(g12, X, ldx, rows, p, sgn, work, ps, s); break;
        default: e = cudaErrorNotSupported; break;
        }
    } else switch (p.n[2]) {
    case 12: e = launch_p12<12>(g12, sm12, X, ldx, rows, p, tw, work, ps, s); break;
    case 16: e = launch_p12<16>(g12, sm12, X, ldx, rows, p, tw, work, ps, s); break;
    case 18: e = launch_p12<18>(g12, sm12, X, ldx, rows, p, tw, work, ps, s); break;
    case 20: e = launch_p12<20>(g12, sm12, X, ldx, rows, p, tw, work, ps, s); break;
    case 24: e = launch_p12<24>(g12, sm12, X, ldx, rows, p, tw, work, ps, s); break;
    case 27: e = launch_p12<27>(g12, sm12, X, ldx, rows, p, tw, work, ps, s); break;
    case 30: e = launch_p12<30>(g12, sm12, X, ldx, rows, p, tw, work, ps, s); break;
    case 32: e = launch_p12<32>(g12, sm12, X, ldx, rows, p, tw, work, ps, s); break;
    case 36: e = launch_p12<36>(g12, sm12, X, ldx, rows, p, tw, work, ps, s); break;
    default: e = launch_p12<0>(g12, sm12, X, ldx, rows, p, tw, work, ps, s); break;
    }
    if (e != cudaSuccess)
        return e;
    // stage 3: constant twiddles where n1 allows, else the paired form (every CTA resident, four per
    // SM, looping over rows) or the plain one
    const bool cst3 = const_twiddles && p.np1 > 0 && p12c_compiled(p.n[0]) && 2 * p.k1 < p.n[0] && p.cd <= 256 &&
                      p3c_smem(p.n[0], p.cd, p.k1, p.ng) <= DFT_SMEM_MAX;
    if (cst3) {
        const size_t sm = p3c_smem(p.n[0], p.cd, p.k1, p.ng);
        const int R = p3c_rows(p.cd), nthr = R * p3c_cdp(p.cd);
        const int per_sm = std::max(1, std::min(4, (int)((200 * 1024) / sm)));  // resident CTAs per SM
        const int g3c = (int)std::min<long long>((rows + R - 1) / R, 152LL * per_sm);
        switch (p.n[0]) {
        case 12: e = launch_p3c<12>(g3c, nthr, sm, work, rows, p, sgn, Y, ldy, s); break;
        case 16: e = launch_p3c<16>(g3c, nthr, sm, work, rows, p, sgn, Y, ldy, s); break;
        case 18: e = launch_p3c<18>(g3c, nthr, sm, work, rows, p, sgn, Y, ldy, s); break;
        case 20: e = launch_p3c<20>(g3c, nthr, sm, work, rows, p, sgn, Y, ldy, s); break;
        case 24: e = launch_p3c<24>(g3c, nthr, sm, work, rows, p, sgn, Y, ldy, s); break;
        case 27: e = launch_p3c<27>(g3c, nthr, sm, work, rows, p, sgn, Y, ldy, s); break;
        default: e = cudaErrorNotSupported; break;
        }
        count_launches(2);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    const int g3 = std::min(rows, paired3 ? 152 * 4 : 152 * 8);
    if (paired3)
        dft_stage3_paired_kernel<<<g3, 256, sm3, s>>>(work, rows, p.n[0], p.cd, p.np1, p.k1, p.ng, p.pair1, tw, Y,
                                                      ldy);
    else
        dft_stage3_kernel<<<g3, 256, sm3, s>>>(work, rows, p.n[0], p.cd, p.ng, p.gmap, tw, Y, ldy);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_dft_rows_ws(const float2 *X, long long ldx, int rows, float2 *Y, long long ldy, const DftPlan &p,
                               float2 *work, cudaStream_t s, bool negative_exponent, bool const_twiddles)
{
    return dft_two_kernel(X, ldx, rows, Y, ldy, p, work, s, negative_exponent, nullptr, const_twiddles);
}

cudaError_t launch_dft_pairs_ws(const float2 *psi, long long nr, const float *sw, int nv, int nc, float2 *Y,
                                long long ldy, const DftPlan &p, float2 *work, cudaStream_t s, bool negative_exponent,
                                int c0, bool const_twiddles)
{
    const PairSrc ps{sw, nv, nc, c0 < 0 ? nv : c0};
    return dft_two_kernel(psi, nr, nv * nc, Y, ldy, p, work, s, negative_exponent, &ps, const_twiddles);
}

cudaError_t launch_dft_rows(const float2 *X, long long ldx, int rows, float2 *Y, long long ldy, const DftPlan &p,
                            cudaStream_t s, bool negative_exponent)
{
    const float2 *tw = negative_exponent ? p.twc : p.tw;
    if (rows <= 0)
        return cudaSuccess;
    if (!dft_supported(p))
        return cudaErrorInvalidValue;
    switch (rows_per_cta(p)) {
    case 4:
        return launch_dft_R<4>(X, ldx, rows, Y, ldy, p, s, tw);
    case 2:
        return launch_dft_R<2>(X, ldx, rows, Y, ldy, p, s, tw);
    default:
        return launch_dft_R<1>(X, ldx, rows, Y, ldy, p, s, tw);
    }
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
