// Sphere transform of whole rows in one kernel (the two FFT phases of Sec. 4.1, pruned to the
// sphere), for grids whose planes and rows allow 16-byte bulk copies.
//
// For every input row x(r), r = (j1 n2 + j2) n3 + j3, the kernel produces
//     y(G) = sum_r x(r) exp(s 2 pi i (m1 j1/n1 + m2 j2/n2 + m3 j3/n3))   for G = m in the sphere
// (s = +1, or -1 with the negative exponent), axis by axis in the order j1, j2, j3:
//   stage A (j1 -> m1): a1[m1][j2][j3] for every |m1| <= M, M = max |m| of the sphere;
//   stage B (j2 -> m2): b[(m1, m2)][j3] for the disk m1^2 + m2^2 <= max of the sphere;
//   stage C (j3 -> m3): y(G) for the sphere points.
// Stage A goes first because it streams: one warp of the CTA copies the row plane by plane (one
// j1 at a time, n2 n3 contiguous values) into a ring of shared-memory slots with 1-D bulk copies,
// and each compute thread owns columns (j2, j3) of the plane, reading its values from consecutive
// shared-memory words and accumulating in registers.  The row of P is read from HBM once and no
// intermediate goes back to global memory.
//
// Every stage pairs the inputs j and n - j (s_j = x_j + x_{n-j}, t_j = x_j - x_{n-j}):
//     sum_j x_j e(s m j / n) = C_m + i S_m,   sum_j x_j e(-s m j / n) = C_m - i S_m,
//     C_m = x_0 + (-1)^m x_{n/2} + sum_{0<j<n/2} s_j cos(2 pi m j/n),  S_m = s sum_{0<j<n/2} t_j sin(2 pi m j/n),
// so one cosine and one sine sum give m and -m.  For stage A the copies arrive in the order
// j1 = 0, n1/2, 1, n1 - 1, 2, n1 - 2, ... so each pair is in shared memory together.
//
// Pair-density rows (the g-space route): row k is f_k(r) = conj(psi_v(r)) psi_c(r) w_k, k = v nc + c,
// and each slot holds plane j1 of psi_c and of psi_v; the product is formed while the plane is read.
//
// Every wait is bounded (the context's limit); a CTA that runs out records GW_E_TIMEOUT, its
// compute warps leave together after a barrier vote, and the copy warp drains its copies before
// the CTA exits.
#include <algorithm>
#include <array>
#include <cmath>
#include <vector>

#include "gw_internal.cuh"
#include "ptx.cuh"

namespace gw {

namespace {

constexpr int FT_COMPUTE = 512;          // compute threads (16 warps: latency hiding for stage A)
constexpr int FT_THREADS = FT_COMPUTE + 32;  // + one copy warp
constexpr uint64_t FT_DRAIN_NS = 2000000000ull;
constexpr int RP = 4;                    // plane pairs per round of stage A

struct FusedArgs {
    const float2 *X;   // rows [rows][ldx], or the states psi [nb][ldx] for pair rows
    long long ldx;
    int rows;
    float2 *Y;
    long long ldy;
    int n1, n2, n3, M, cd, ng, slots;
    const int *tab;    // the plan's integer tables (FusedPlan::layout)
    const float2 *tw;  // [n1][M+1] | [n2][M+1] | [n3][M+1]: (cos, sin) of 2 pi m j / n_a
    float sgn;         // +1: exp(+i...), -1: exp(-i...)
    const float *sw;   // pair rows: weights of the pairs (null: plain rows)
    int nv, nc, c0;
    uint32_t *err;
    uint64_t wait_ns;
    // byte offsets in dynamic shared memory
    unsigned o_a1, o_b, o_y, o_tw, o_tab, o_bar;
    unsigned slot_bytes;
    int ntab, ntw;
};

// integer tables, each [entries] ints:
//   m2max[2M+1]           max |m2| of the disk at m1 = i1 - M
//   d12[(2M+1)^2]         disk index of (m1, m2) = (i1 - M, i2 - M), or -1
//   m3max[cd]             max |m3| of the sphere at disk point d
//   gidx[cd][2M+1]        sphere index of (m1, m2, m3 = i3 - M) of disk point d, or -1
__host__ __device__ inline int tab_m2max(int) { return 0; }
__host__ __device__ inline int tab_d12(int M) { return 2 * M + 1; }
__host__ __device__ inline int tab_m3max(int M) { return tab_d12(M) + (2 * M + 1) * (2 * M + 1); }
__host__ __device__ inline int tab_gidx(int M, int cd) { return tab_m3max(M) + cd; }
__host__ __device__ inline int tab_size(int M, int cd) { return tab_gidx(M, cd) + cd * (2 * M + 1); }

__device__ __forceinline__ void named_bar1()
{
    asm volatile("bar.sync 1, %0;" ::"r"(FT_COMPUTE) : "memory");
}

// barrier over the compute threads that also ORs a predicate across them
__device__ __forceinline__ bool named_bar1_or(bool p)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\t"
        "setp.ne.u32 pi, %1, 0;\n\t"
        "bar.red.or.pred po, 1, %2, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(FT_COMPUTE)
        : "memory");
    return r != 0;
}

// j1 of the q-th plane of a row: 0, n/2 (even n), then 1, n-1, 2, n-2, ...
__device__ __forceinline__ int plane_order(int q, int n)
{
    const int head = (n % 2 == 0) ? 2 : 1;
    if (q == 0)
        return 0;
    if (q == 1 && head == 2)
        return n / 2;
    const int p = q - head;  // pair index p/2, member p%2
    const int j = 1 + p / 2;
    return (p & 1) ? n - j : j;
}

__device__ __forceinline__ float2 pair_density(float2 a, float2 b, float w)  // conj(a) b w
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y) * w, fmaf(a.x, b.y, -a.y * b.x) * w);
}

template <int CPT, int MM, bool PAIR>
__global__ void __launch_bounds__(FT_THREADS, 1) dft_fused_kernel(const FusedArgs a)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const int P = a.n2 * a.n3;
    const int M = a.M;
    float2 *a1 = reinterpret_cast<float2 *>(smem + a.o_a1);  // [2M+1][P]
    float2 *bb = reinterpret_cast<float2 *>(smem + a.o_b);   // [cd][n3 + 1]
    float2 *yy = reinterpret_cast<float2 *>(smem + a.o_y);   // [ng]
    float2 *tw = reinterpret_cast<float2 *>(smem + a.o_tw);
    int *tab = reinterpret_cast<int *>(smem + a.o_tab);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + a.o_bar);
    uint64_t *empty = full + a.slots;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + a.slots);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int t = tid; t < a.ntw; t += FT_THREADS)
        tw[t] = a.tw[t];
    for (int t = tid; t < a.ntab; t += FT_THREADS)
        tab[t] = a.tab[t];
    if (tid == 0) {
        for (int s = 0; s < a.slots; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], FT_COMPUTE / 32);
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    const float2 *twA = tw, *twB = tw + a.n1 * (M + 1), *twC = twB + a.n2 * (M + 1);
    const int *m2max = tab + tab_m2max(M), *d12 = tab + tab_d12(M), *m3max = tab + tab_m3max(M);
    const int *gidx = tab + tab_gidx(M, a.cd);
    const unsigned plane_bytes = (unsigned)P * sizeof(float2);

    if (warp == FT_COMPUTE / 32) {
        // ---------------- copy warp: planes of this CTA's rows, in stage A's order, into the ring
        if (lane == 0) {
            // ring position of the next copy, advanced without division: slot, its pass parity, and
            // whether the ring has wrapped once (from then on a slot must be freed before reuse)
            int slot = 0, par = 0, issued = 0;
            bool stop = false;
            for (int row = blockIdx.x; row < a.rows && !stop; row += gridDim.x) {
                const float2 *src_c = a.X + (size_t)row * a.ldx, *src_v = nullptr;
                if (PAIR) {
                    const int v = row / a.nc;
                    src_c = a.X + (size_t)(a.c0 + row - v * a.nc) * a.ldx;
                    src_v = a.X + (size_t)v * a.ldx;
                }
                for (int qq = 0; qq < a.n1; ++qq) {
                    const int s = slot;
                    if (issued >= a.slots && !mbar_wait(&empty[s], (uint32_t)(par ^ 1), a.wait_ns)) {
                        record_error(a.err, GW_E_TIMEOUT, SITE_HERK_PRODUCER, blockIdx.x);
                        *abort_flag = 1;
                        stop = true;
                        break;
                    }
                    if (*abort_flag) {
                        stop = true;
                        break;
                    }
                    const int j1 = plane_order(qq, a.n1);
                    uint8_t *dst = smem + (size_t)s * a.slot_bytes;
                    mbar_arrive_expect_tx(&full[s], PAIR ? 2 * plane_bytes : plane_bytes);
                    bulk_g2s(dst, src_c + (size_t)j1 * P, plane_bytes, &full[s]);
                    if (PAIR)
                        bulk_g2s(dst + plane_bytes, src_v + (size_t)j1 * P, plane_bytes, &full[s]);
                    ++issued;
                    if (++slot == a.slots) {
                        slot = 0;
                        par ^= 1;
                    }
                }
            }
            // drain: no copy of this CTA may still be landing when it exits (the last min(issued,
            // slots) copies, walked backwards from the next ring position)
            for (int k = 0; k < min(issued, a.slots); ++k) {
                if (--slot < 0) {
                    slot = a.slots - 1;
                    par ^= 1;
                }
                if (!mbar_wait(&full[slot], (uint32_t)par, FT_DRAIN_NS)) {
                    record_error(a.err, GW_E_TIMEOUT, SITE_HERK_DRAIN, blockIdx.x);
                    break;
                }
            }
        }
        __syncwarp();
    } else {
        // ---------------- compute warps
        const float sgn = a.sgn;
        int slot = 0, par = 0;  // ring position of the next plane (as in the copy warp)
        bool failed = false;
        for (int row = blockIdx.x; row < a.rows; row += gridDim.x) {
            const float w = PAIR ? a.sw[row] : 1.0f;
            // stage A: C_m, S_m of every owned column over j1 (paired planes)
            float2 C[CPT][MM + 1], S[CPT][MM + 1];
#pragma unroll
            for (int c = 0; c < CPT; ++c)
#pragma unroll
                for (int m = 0; m <= MM; ++m) {
                    C[c][m] = make_float2(0.f, 0.f);
                    S[c][m] = make_float2(0.f, 0.f);
                }
            // Rounds: first the planes without a partner (j1 = 0, and n1/2 for even n1), then up to
            // RP pairs (j, n1 - j) at a time, so every wait and release covers several planes and
            // each thread has many independent multiply-adds between them.
            const int nsingle = (a.n1 % 2 == 0) ? 2 : 1;
            for (int pos = 0; pos < a.n1;) {
                const bool singles = pos == 0;
                const int np = singles ? 0 : min(RP, (a.n1 - pos) / 2);  // pairs in this round
                const int take = singles ? nsingle : 2 * np;
                int su[2 * RP], pu[2 * RP];
                {
                    int sl = slot, pa = par;
#pragma unroll
                    for (int u = 0; u < 2 * RP; ++u) {
                        su[u] = sl;
                        pu[u] = pa;
                        if (u < take && ++sl == a.slots) {
                            sl = 0;
                            pa ^= 1;
                        }
                    }
                    slot = sl;
                    par = pa;
                }
#pragma unroll
                for (int u = 0; u < 2 * RP; ++u)
                    if (u < take && !failed && !mbar_wait(&full[su[u]], (uint32_t)pu[u], a.wait_ns)) {
                        if (lane == 0)
                            record_error(a.err, GW_E_TIMEOUT, SITE_HERK_MMA, blockIdx.x);
                        failed = true;
                    }
                failed = __any_sync(0xffffffffu, failed);
                if (!failed) {
                    if (singles) {
                        // cos = 1 (j1 = 0) or (-1)^m (j1 = n1/2), sin = 0
                        for (int u = 0; u < nsingle; ++u) {
                            const float2 *xs = reinterpret_cast<const float2 *>(smem + (size_t)su[u] * a.slot_bytes);
#pragma unroll
                            for (int c = 0; c < CPT; ++c) {
                                const int col = tid + FT_COMPUTE * c;
                                if (col < P) {
                                    float2 x0 = xs[col];
                                    if (PAIR)
                                        x0 = pair_density(xs[P + col], x0, w);
#pragma unroll
                                    for (int m = 0; m <= MM; ++m)
                                        if (m <= M) {
                                            const float sg = (u == 1 && (m & 1)) ? -1.f : 1.f;
                                            C[c][m].x = fmaf(sg, x0.x, C[c][m].x);
                                            C[c][m].y = fmaf(sg, x0.y, C[c][m].y);
                                        }
                                }
                            }
                        }
                    } else {
                        const int j0 = 1 + (pos - nsingle) / 2;  // j of the round's first pair
#pragma unroll
                        for (int pp = 0; pp < RP; ++pp)
                            if (pp < np) {
                                const float2 *x0s = reinterpret_cast<const float2 *>(smem + (size_t)su[2 * pp] * a.slot_bytes);
                                const float2 *x1s =
                                    reinterpret_cast<const float2 *>(smem + (size_t)su[2 * pp + 1] * a.slot_bytes);
                                const float2 *cs = twA + (j0 + pp) * (M + 1);
#pragma unroll
                                for (int c = 0; c < CPT; ++c) {
                                    const int col = tid + FT_COMPUTE * c;
                                    if (col < P) {
                                        float2 x0 = x0s[col], x1 = x1s[col];
                                        if (PAIR) {
                                            x0 = pair_density(x0s[P + col], x0, w);
                                            x1 = pair_density(x1s[P + col], x1, w);
                                        }
                                        const float2 sp = make_float2(x0.x + x1.x, x0.y + x1.y);
                                        const float2 tp = make_float2(x0.x - x1.x, x0.y - x1.y);
#pragma unroll
                                        for (int m = 0; m <= MM; ++m)
                                            if (m <= M) {
                                                const float2 t = cs[m];
                                                C[c][m].x = fmaf(sp.x, t.x, C[c][m].x);
                                                C[c][m].y = fmaf(sp.y, t.x, C[c][m].y);
                                                if (m > 0) {  // sin(0) = 0
                                                    S[c][m].x = fmaf(tp.x, t.y, S[c][m].x);
                                                    S[c][m].y = fmaf(tp.y, t.y, S[c][m].y);
                                                }
                                            }
                                    }
                                }
                            }
                    }
                }
                __syncwarp();
                if (lane == 0 && !failed)
                    for (int u = 0; u < take; ++u)
                        mbar_arrive(&empty[su[u]]);
                pos += take;
            }
            // results of stage A: a1[M +- m][col] = C_m +- i sgn S_m
            if (!failed) {
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    const int col = tid + FT_COMPUTE * c;
                    if (col < P) {
#pragma unroll
                        for (int m = 0; m <= MM; ++m)
                            if (m <= M) {
                                const float2 cc = C[c][m], ss = make_float2(sgn * S[c][m].x, sgn * S[c][m].y);
                                a1[(size_t)(M + m) * P + col] = make_float2(cc.x - ss.y, cc.y + ss.x);
                                if (m > 0)
                                    a1[(size_t)(M - m) * P + col] = make_float2(cc.x + ss.y, cc.y - ss.x);
                            }
                    }
                }
            }
            if (named_bar1_or(failed || *abort_flag != 0)) {
                if (tid == 0)
                    *abort_flag = 1;
                break;
            }
            // stage B: items (i1, j3), sums over j2 for |m2| <= m2max[i1]
            const int nB = (2 * M + 1) * a.n3;
            for (int t = tid; t < nB; t += FT_COMPUTE) {
                const int i1 = t / a.n3, j3 = t - i1 * a.n3;
                const int M2 = m2max[i1];
                const float2 *col = a1 + (size_t)i1 * P + j3;
                float2 Cb[MM + 1], Sb[MM + 1];
                const float2 z0 = col[0];
#pragma unroll
                for (int m = 0; m <= MM; ++m) {
                    Cb[m] = z0;
                    Sb[m] = make_float2(0.f, 0.f);
                }
                if (a.n2 % 2 == 0) {
                    const float2 zh = col[(size_t)(a.n2 / 2) * a.n3];
#pragma unroll
                    for (int m = 0; m <= MM; ++m) {
                        const float sg = (m & 1) ? -1.f : 1.f;
                        Cb[m].x = fmaf(sg, zh.x, Cb[m].x);
                        Cb[m].y = fmaf(sg, zh.y, Cb[m].y);
                    }
                }
                for (int j2 = 1; 2 * j2 < a.n2; ++j2) {
                    const float2 u = col[(size_t)j2 * a.n3], v = col[(size_t)(a.n2 - j2) * a.n3];
                    const float2 sp = make_float2(u.x + v.x, u.y + v.y), tp = make_float2(u.x - v.x, u.y - v.y);
#pragma unroll
                    for (int m = 0; m <= MM; ++m)
                        if (m <= M2) {
                            const float2 cs = twB[j2 * (M + 1) + m];
                            Cb[m].x = fmaf(sp.x, cs.x, Cb[m].x);
                            Cb[m].y = fmaf(sp.y, cs.x, Cb[m].y);
                            Sb[m].x = fmaf(tp.x, cs.y, Sb[m].x);
                            Sb[m].y = fmaf(tp.y, cs.y, Sb[m].y);
                        }
                }
                const int *drow = d12 + i1 * (2 * M + 1);
#pragma unroll
                for (int m = 0; m <= MM; ++m)
                    if (m <= M2) {
                        const float2 ss = make_float2(sgn * Sb[m].x, sgn * Sb[m].y);
                        bb[(size_t)drow[M + m] * (a.n3 + 1) + j3] = make_float2(Cb[m].x - ss.y, Cb[m].y + ss.x);
                        if (m > 0)
                            bb[(size_t)drow[M - m] * (a.n3 + 1) + j3] = make_float2(Cb[m].x + ss.y, Cb[m].y - ss.x);
                    }
            }
            named_bar1();
            // stage C: one disk point per item, sums over j3 for |m3| <= m3max[d]
            for (int d = tid; d < a.cd; d += FT_COMPUTE) {
                const int M3 = m3max[d];
                const float2 *col = bb + (size_t)d * (a.n3 + 1);
                float2 Cc[MM + 1], Sc[MM + 1];
                const float2 z0 = col[0];
#pragma unroll
                for (int m = 0; m <= MM; ++m) {
                    Cc[m] = z0;
                    Sc[m] = make_float2(0.f, 0.f);
                }
                if (a.n3 % 2 == 0) {
                    const float2 zh = col[a.n3 / 2];
#pragma unroll
                    for (int m = 0; m <= MM; ++m) {
                        const float sg = (m & 1) ? -1.f : 1.f;
                        Cc[m].x = fmaf(sg, zh.x, Cc[m].x);
                        Cc[m].y = fmaf(sg, zh.y, Cc[m].y);
                    }
                }
                for (int j3 = 1; 2 * j3 < a.n3; ++j3) {
                    const float2 u = col[j3], v = col[a.n3 - j3];
                    const float2 sp = make_float2(u.x + v.x, u.y + v.y), tp = make_float2(u.x - v.x, u.y - v.y);
#pragma unroll
                    for (int m = 0; m <= MM; ++m)
                        if (m <= M3) {
                            const float2 cs = twC[j3 * (M + 1) + m];
                            Cc[m].x = fmaf(sp.x, cs.x, Cc[m].x);
                            Cc[m].y = fmaf(sp.y, cs.x, Cc[m].y);
                            Sc[m].x = fmaf(tp.x, cs.y, Sc[m].x);
                            Sc[m].y = fmaf(tp.y, cs.y, Sc[m].y);
                        }
                }
                const int *grow = gidx + (size_t)d * (2 * M + 1);
#pragma unroll
                for (int m = 0; m <= MM; ++m)
                    if (m <= M3) {
                        const float2 ss = make_float2(sgn * Sc[m].x, sgn * Sc[m].y);
                        yy[grow[M + m]] = make_float2(Cc[m].x - ss.y, Cc[m].y + ss.x);
                        if (m > 0)
                            yy[grow[M - m]] = make_float2(Cc[m].x + ss.y, Cc[m].y - ss.x);
                    }
            }
            named_bar1();
            float2 *yrow = a.Y + (size_t)row * a.ldy;
            for (int g = tid; g < a.ng; g += FT_COMPUTE)
                yrow[g] = yy[g];
            // the next row's stage A ends in a barrier before a1, b or y are written again
        }
    }
    __syncthreads();
}

template <int CPT, int MM, bool PAIR>
cudaError_t launch_t(const FusedArgs &a, size_t smem, int grid, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(dft_fused_kernel<CPT, MM, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    dft_fused_kernel<CPT, MM, PAIR><<<grid, FT_THREADS, smem, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

size_t align128(size_t x)
{
    return (x + 127) & ~(size_t)127;
}

}  // namespace

// Host plan: tables and twiddles from the sphere (in basis order) of an n1 x n2 x n3 grid.
bool FusedPlan::build(const int n_[3], const std::vector<std::array<int, 3>> &g)
{
    ok = false;
    for (int a = 0; a < 3; ++a)
        n[a] = n_[a];
    ng = static_cast<int>(g.size());
    M = 0;
    for (const auto &v : g)
        for (int a = 0; a < 3; ++a)
            M = std::max(M, std::abs(v[a]));
    for (int a = 0; a < 3; ++a)
        if (2 * M >= n[a])
            return false;  // +-m must be distinct on every axis
    const int W = 2 * M + 1;
    // disk (m1, m2) and, per disk point, the m3 of the sphere; the sphere must be symmetric in
    // each component (it is, for |m|^2 <= gcut) and its m2, m3 ranges contiguous
    std::vector<std::vector<int>> gi(W * W, std::vector<int>(W, -1));
    for (int i = 0; i < ng; ++i)
        gi[(g[i][0] + M) * W + g[i][1] + M][g[i][2] + M] = i;
    tab.assign(0, 0);
    std::vector<int> m2max(W, -1), d12(W * W, -1), m3max, gidx;
    cd = 0;
    for (int i1 = 0; i1 < W; ++i1)
        for (int i2 = 0; i2 < W; ++i2) {
            const auto &col = gi[i1 * W + i2];
            int M3 = -1;
            for (int i3 = 0; i3 < W; ++i3)
                if (col[i3] >= 0)
                    M3 = std::max(M3, std::abs(i3 - M));
            if (M3 < 0)
                continue;
            for (int m3 = -M3; m3 <= M3; ++m3)
                if (col[m3 + M] < 0)
                    return false;  // m3 range not contiguous
            d12[i1 * W + i2] = cd++;
            m3max.push_back(M3);
            for (int i3 = 0; i3 < W; ++i3)
                gidx.push_back(col[i3]);
            m2max[i1] = std::max(m2max[i1], std::abs(i2 - M));
        }
    for (int i1 = 0; i1 < W; ++i1) {
        if (m2max[i1] < 0)
            return false;
        for (int m2 = -m2max[i1]; m2 <= m2max[i1]; ++m2)
            if (d12[i1 * W + m2 + M] < 0)
                return false;  // m2 range not contiguous
        for (int m2 = -m2max[i1]; m2 <= m2max[i1]; ++m2)
            if (d12[i1 * W + M - m2] < 0)
                return false;
    }
    tab.reserve(tab_size(M, cd));
    tab.insert(tab.end(), m2max.begin(), m2max.end());
    tab.insert(tab.end(), d12.begin(), d12.end());
    tab.insert(tab.end(), m3max.begin(), m3max.end());
    tab.insert(tab.end(), gidx.begin(), gidx.end());
    tw.clear();
    for (int a = 0; a < 3; ++a)
        for (int j = 0; j < n[a]; ++j)
            for (int m = 0; m <= M; ++m) {
                const double ph = 2.0 * 3.14159265358979323846 * (double)((long)m * j % n[a]) / n[a];
                tw.push_back(make_float2((float)std::cos(ph), (float)std::sin(ph)));
            }
    ok = true;
    return true;
}

size_t FusedPlan::device_bytes() const
{
    return align128(tab.size() * sizeof(int)) + tw.size() * sizeof(float2);
}

cudaError_t FusedPlan::upload(void *dev, cudaStream_t s)
{
    d_tab = static_cast<int *>(dev);
    d_tw = reinterpret_cast<float2 *>(static_cast<uint8_t *>(dev) + align128(tab.size() * sizeof(int)));
    cudaError_t e = cudaMemcpyAsync(d_tab, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);  // the host vectors stay, but keep uploads ordered before use
    return e;
}

cudaError_t launch_dft_fused(const float2 *X, long long ldx, int rows, float2 *Y, long long ldy, const FusedPlan &p,
                             bool negative_exponent, const float *sw, int nv, int nc, int c0, uint32_t *err,
                             uint64_t wait_ns, cudaStream_t s)
{
    if (rows <= 0)
        return cudaSuccess;
    if (!p.ok || !p.d_tab)
        return cudaErrorNotSupported;
    const int P = p.n[1] * p.n[2];
    const bool pair = sw != nullptr;
    // 16-byte bulk copies: planes, rows and the base must be 16-byte aligned
    if (P % 2 != 0 || ldx % 2 != 0 || (reinterpret_cast<size_t>(X) & 15) != 0)
        return cudaErrorNotSupported;
    const int cpt = (P + FT_COMPUTE - 1) / FT_COMPUTE;
    const int MM = p.M <= 4 ? 4 : p.M <= 6 ? 6 : p.M <= 8 ? 8 : 0;
    if (MM == 0 || cpt > 2)
        return cudaErrorNotSupported;
    FusedArgs a{};
    a.X = X;
    a.ldx = ldx;
    a.rows = rows;
    a.Y = Y;
    a.ldy = ldy;
    a.n1 = p.n[0];
    a.n2 = p.n[1];
    a.n3 = p.n[2];
    a.M = p.M;
    a.cd = p.cd;
    a.ng = p.ng;
    a.tab = p.d_tab;
    a.tw = p.d_tw;
    a.sgn = negative_exponent ? -1.f : 1.f;
    a.sw = sw;
    a.nv = nv;
    a.nc = nc;
    a.c0 = c0;
    a.err = err;
    a.wait_ns = wait_ns;
    a.ntab = (int)p.tab.size();
    a.ntw = (int)p.tw.size();
    const size_t plane = (size_t)P * sizeof(float2);
    a.slot_bytes = (unsigned)align128(pair ? 2 * plane : plane);
    // shared memory: the ring, then a1, b, y, twiddles, tables, barriers.  One CTA per SM (the
    // compute threads' registers allow no second one), so the ring takes what is left of the SM's
    // shared memory: the planes in flight must cover the HBM latency (about 2 us x 44 GB/s per SM).
    const size_t fixed = align128(sizeof(float2) * (size_t)(2 * p.M + 1) * P) +
                         align128(sizeof(float2) * (size_t)p.cd * (p.n[2] + 1)) + align128(sizeof(float2) * p.ng) +
                         align128(sizeof(float2) * p.tw.size()) + align128(sizeof(int) * p.tab.size());
    const size_t cap = 227 * 1024;
    auto total = [&](int slots) { return fixed + (size_t)slots * a.slot_bytes + align128((size_t)slots * 16 + 16); };
    int slots = 64;
    while (slots > 3 && total(slots) > cap)
        --slots;
    if (total(slots) > cap)
        return cudaErrorNotSupported;
    a.slots = slots;
    size_t o = (size_t)slots * a.slot_bytes;
    a.o_a1 = (unsigned)o;
    o += align128(sizeof(float2) * (size_t)(2 * p.M + 1) * P);
    a.o_b = (unsigned)o;
    o += align128(sizeof(float2) * (size_t)p.cd * (p.n[2] + 1));
    a.o_y = (unsigned)o;
    o += align128(sizeof(float2) * p.ng);
    a.o_tw = (unsigned)o;
    o += align128(sizeof(float2) * p.tw.size());
    a.o_tab = (unsigned)o;
    o += align128(sizeof(int) * p.tab.size());
    a.o_bar = (unsigned)o;
    o += align128((size_t)slots * 16 + 16);
    const size_t smem = o;
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
    const int grid = std::max(1, std::min(rows, nsm));
    if (pair) {
        if (cpt <= 1 && MM == 4) return launch_t<1, 4, true>(a, smem, grid, s);
        if (cpt <= 2 && MM <= 6) return launch_t<2, 6, true>(a, smem, grid, s);
        if (cpt <= 2 && MM <= 8) return launch_t<2, 8, true>(a, smem, grid, s);
    } else {
        if (cpt <= 1 && MM == 4) return launch_t<1, 4, false>(a, smem, grid, s);
        if (cpt <= 2 && MM <= 6) return launch_t<2, 6, false>(a, smem, grid, s);
        if (cpt <= 2 && MM <= 8) return launch_t<2, 8, false>(a, smem, grid, s);
    }
    return cudaErrorNotSupported;
}

}  // namespace gw
