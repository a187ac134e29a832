// Complex GEMM C = A B on the 16-bit tensor cores from sliced FP64 operands, and the Newton
// iteration X <- X (2I - eps X) of Sec. 5.1 for eps^-1 built on it.
//
// FP64 runs at about 1 TFLOP/s on this GPU and FP16 tensor MMAs at about 2 PFLOP/s, so the
// inverse is carried by the tensor cores:
//  * Phase 1: Newton iterations whose products use the FP16X3 split (22 significant bits), until
//    max |I - eps X| < 3e-5, from the Jacobi-scaled start X0 = 2 / (1 + u) D^-1: D = diag(eps)
//    (through rs_i = 1 / sqrt(eps_ii) in FP32, D^-1 = diag(rs^2)) and
//    u = max_i rs_i sum_j |eps_ij| rs_j >= lambda_max(D^-1/2 eps D^-1/2).  eps X0 is similar to
//    2 / (1 + u) D^-1/2 eps D^-1/2, whose eigenvalues lie in (0, 2) for a Hermitian positive
//    definite eps, and the error e = I - eps X squares each step.  Scaling the rows and columns of
//    eps by a positive diagonal leaves the scaled matrix, and so the step count, unchanged.  A
//    diagonal entry that is not positive and finite falls back to X0 = 2 / (1 + u) I with the
//    plain row-sum bound u = max_i sum_j |eps_ij|.
//  * Phase 2: up to three refinement steps R = I - eps X, X <- X + X R.  R is computed to FP64 accuracy
//    from integer slices (the error-free splitting of Ozaki, Ogita, Oishi and Rump, Numer.
//    Algorithms 59, 2012): every entry scaled into [-1, 1] is a sum of slices a_t 2^(-6(t+1))
//    with integer a_0 in [-64, 64] and a_t in [-32, 32] (t >= 1); nine slices keep 54 bits.  The
//    slice products a_t b_u are exact in FP16 and their sums over one work slot stay below 2^24,
//    so the FP32 tensor-core accumulation is exact; the slots are scaled by 2^(-6(t+u+2)) and
//    added in FP64.  X R only needs the relative accuracy of the FP16X3 split, because R is small.
//    Each refinement squares the residual (plus the FP16X3 error of X R, ~4e-6 |R|); once a
//    measured residual is <= 1e-9 its correction is the last one (the result then sits near 4e-15).
//    If three refinements end with a last measured residual above 1e-8 (or a non-finite one), the
//    inverse is reported as GW_E_NUMERIC.
//
// Operand planes (K-major, 8-row x 16-byte core matrices, as in the rank-k update): element
// (r, k) of plane p sits at 16-bit offset ((kc Rpad/128 + r/128) NP + p) 2048 + ((r%128)/8) 128 +
// ((k%16)/8) 64 + (r%8) 8 + k%8 with kc = k / 16: the NP planes of one chunk of one 128-row block
// are contiguous, so a stage arrives in one bulk copy per operand (large copies reach a higher
// per-SM ingress than 4 KB ones).  A operand (row i of A, k along the row): planes 2t (Re) and
// 2t + 1 (Im) of slice t.  B operand (row j = column j of B, k down the column): planes 2t (Re)
// and 2t + 1 (Im), so the 256 rows starting at Re are [Re; Im].  Then one M = 128, N = 256 MMA with
// A = Re(A) adds Re A Re B into the Re columns of the accumulator and Re A Im B into its Im
// columns, and two N = 128 MMAs with A = Im(A) add -Im A Im B (the A-negate bit of the instruction
// descriptor) into the Re columns and Im A Re B into the Im columns: C = A B with the tensor work of
// two N = 256 MMAs per slice pair and 16-wide chunk, and no negated plane in memory.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "gw_internal.cuh"
#include "ptx.cuh"

namespace gw {

namespace {

constexpr int ZT = 128;
constexpr uint32_t ZPL = ZT * 16 * 2;       // 4 KB: one plane of one 128-row block, one chunk
// A stage is one chunk of one slice pair (A Re, A Im, B Re, B Im: 16 KB, three MMAs) for the
// integer slices, and one chunk of all three FP16X3 pairs (A hi Re, Im, A lo Re, Im, B hi Re, Im,
// B lo Re, Im: 32 KB, nine MMAs, one commit) for the split, where each slice then loads once per
// chunk.
constexpr uint32_t ZSTAGE = 4 * ZPL;
constexpr int ZSTAGES = 6;                  // twelve stages in flight per SM cover the copy latency
constexpr uint32_t ZPIPE = ZSTAGES * ZSTAGE;  // 96 KB: two CTAs per SM
constexpr uint32_t ZSTAGE3 = 8 * ZPL;
constexpr int ZSTAGES3 = 3;
static_assert(ZSTAGES3 * ZSTAGE3 <= ZPIPE, "the fused stages share the pipeline buffers");
static_assert(128 * 65 * 8 <= ZPIPE, "epilogue staging must fit in the pipeline buffers");
constexpr size_t ZSMEM = ZPIPE + 128;
constexpr int ZTHREADS = 192;               // warp 0 copies, warp 1 MMAs, warps 2..5 epilogue
constexpr uint32_t LBO = 128, SBO = 256;
constexpr uint64_t DRAIN_NS = 2000000000ull;

constexpr int MODE_FP16X3 = 0, MODE_SLICES = 1;
constexpr int OZ_SLICES = 9;
constexpr double NS_TOL = 3e-5;     // phase 1 stops below this max |I - eps X|
constexpr double NS_LAST = 1e-9;    // a refinement whose residual is below this is the last one
constexpr double NS_ACCEPT = 1e-8;  // largest residual before the last correction
constexpr int NS_MAX = 16, NS_REFINE = 3;

// Scale exponent e of a matrix from the bits of max(|Re|, |Im|): m (1 + 2^-20) < 2^e, so a max
// taken in FP32 (relative error 2^-24) still bounds every entry (0 for an all-zero or non-finite
// matrix; a non-finite residual is caught by the final check).
__device__ __forceinline__ int exp_of(const unsigned long long *w)
{
    const double m = __longlong_as_double((long long)*w);
    if (!(m > 0.0) || !isfinite(m))
        return 0;
    int e;
    frexp(m * (1.0 + 0x1p-20), &e);
    return e;
}

__device__ __forceinline__ void named_bar_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Named barrier over n threads that also ORs a predicate, so the participants agree on it.
__device__ __forceinline__ bool named_bar_or(int id, int n, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"(pred ? 1u : 0u), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ uint16_t h16(float x)
{
    __half h = __float2half_rn(x);
    return *reinterpret_cast<uint16_t *>(&h);
}

// max(|Re|, |Im|) over a rows x cols complex128 matrix into *w (as the bits of a non-negative
// double, which order like unsigned integers).  *w must be zero (or smaller) beforehand.
__global__ void zmaxabs_kernel(const double2 *__restrict__ M, int rows, int cols, long ld, unsigned long long *w)
{
    __shared__ double red[32];
    double best = 0.0;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    for (int r = blockIdx.y; r < rows && c < cols; r += gridDim.y) {
        const double2 z = M[(size_t)r * ld + c];
        best = fmax(best, fmax(fabs(z.x), fabs(z.y)));
    }
    for (int o = 16; o > 0; o >>= 1)
        best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i)
            best = fmax(best, red[i]);
        atomicMax(w, (unsigned long long)__double_as_longlong(best));
    }
}

// Slice a complex128 matrix into operand planes (layouts above).  One block per (16-wide chunk
// kc, 128-row block rb of the operand): the 16 x 128 tile goes through shared memory, so both
// orientations read contiguous runs of M and every plane is written in 4 KB runs.  transpose = 0:
// operand row r is row r of M (A operand, element (r, k) = M[r][k]); transpose = 1: operand row r
// is column r of M (B operand, element (r, k) = M[k][r]).  npl = 2 planes (Re, Im) per slice for
// either operand.  Entries outside rows x K are zero.
//   FP16X3: y = float(x) 2^(14 - e), hi = rn16(y), lo = rn16(y - hi).
//   slices: n = rint(x 2^(6 ns - e)) (|n| <= 2^(6 ns)) written in balanced base 64,
//           n = sum_t a_t 2^(6 (ns - 1 - t)): a_(ns-1) .. a_1 in [-32, 31] from the low end, a_0 =
//           the rest, |a_0| <= 64; so x 2^-e = sum_t a_t 2^(-6 (t + 1)) up to 2^(-6 ns - 1).
__global__ void __launch_bounds__(512) zslice_kernel(const double2 *__restrict__ M, long ld, int rows, int K,
                                                     int transpose, int Rpad, int mode, int ns, int npl,
                                                     const unsigned long long *maxw, uint16_t *__restrict__ planes,
                                                     const int *skip)
{
    if (skip && *skip)
        return;
    __shared__ double2 tile[16][129];
    const int kc = blockIdx.x, rb = blockIdx.y;
    const int k0 = kc * 16, r0 = rb * 128;
    const double2 zero = make_double2(0.0, 0.0);
    if (transpose) {
        for (int q = threadIdx.x; q < 2048; q += blockDim.x) {
            const int kk = q >> 7, rr = q & 127, r = r0 + rr, k = k0 + kk;
            tile[kk][rr] = (r < rows && k < K) ? M[(size_t)k * ld + r] : zero;
        }
    } else {
        for (int q = threadIdx.x; q < 2048; q += blockDim.x) {
            const int rr = q >> 4, kk = q & 15, r = r0 + rr, k = k0 + kk;
            tile[kk][rr] = (r < rows && k < K) ? M[(size_t)r * ld + k] : zero;
        }
    }
    // the scales once per block: FP64 work per thread would rival the slicing itself here
    __shared__ float s_scf;
    __shared__ double s_scd;
    if (threadIdx.x == 0) {
        const int e = exp_of(maxw);
        s_scf = ldexpf(1.0f, 14 - e);
        s_scd = ldexp(1.0, 6 * ns - e);
    }
    __syncthreads();
    const int NP = ns * npl;
    constexpr size_t per = 2048;  // consecutive planes of one block and chunk
    uint16_t *base0 = planes + ((size_t)kc * (Rpad / ZT) + rb) * NP * per;
    const float scf = s_scf;
    const double scd = s_scd;
    for (int rem = threadIdx.x; rem < 2048; rem += blockDim.x) {
        const int rr = (rem >> 7) * 8 + ((rem & 63) >> 3);
        const int kk = ((rem & 127) >> 6) * 8 + (rem & 7);
        const double2 z = tile[kk][rr];
        uint16_t *b = base0 + rem;
        if (mode == MODE_FP16X3) {
            const float yr = (float)z.x * scf, yi = (float)z.y * scf;
            const uint16_t rh = h16(yr), ih = h16(yi);
            const uint16_t rl = h16(yr - __half2float(*reinterpret_cast<const __half *>(&rh)));
            const uint16_t il = h16(yi - __half2float(*reinterpret_cast<const __half *>(&ih)));
            const uint16_t re[2] = {rh, rl}, im[2] = {ih, il};
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                b[(size_t)(2 * t) * per] = re[t];
                b[(size_t)(2 * t + 1) * per] = im[t];
            }
        } else {
            long long nr = __double2ll_rn(z.x * scd), ni = __double2ll_rn(z.y * scd);
            for (int t = ns - 1; t >= 0; --t) {
                long long ar, ai;
                if (t > 0) {
                    ar = ((nr + 32) & 63) - 32;
                    ai = ((ni + 32) & 63) - 32;
                    nr = (nr - ar) >> 6;  // exact: nr - ar is a multiple of 64
                    ni = (ni - ai) >> 6;
                } else {
                    ar = nr;
                    ai = ni;
                }
                const uint16_t hr = h16((float)ar), hi = h16((float)ai);  // |a| <= 64: exact
                b[(size_t)(2 * t) * per] = hr;
                b[(size_t)(2 * t + 1) * per] = hi;
            }
        }
    }
}

// One work slot of the sliced product: slice pairs [p0, p1) of the pair list over chunks
// [kc0, kc1); the slot's result is one FP32 complex tile per output tile, T[slot][Mpad][Npad].
struct ZSlot {
    int p0, p1, kc0, kc1;
};

template <bool F3>  // true: FP16X3 slots, one stage per chunk with the pairs (0,0), (0,1), (1,0)
__global__ void __launch_bounds__(ZTHREADS, 2)
    zgemm16_kernel(const uint16_t *__restrict__ Ap, int npA, int Mpad, const uint16_t *__restrict__ Bp, int npB,
                   int Npad, const int2 *__restrict__ pairs, const ZSlot *__restrict__ slots, int ntj,
                   float2 *__restrict__ T, uint32_t *err, uint64_t wait_ns, const int *skip)
{
    constexpr uint32_t SB = F3 ? ZSTAGE3 : ZSTAGE;
    constexpr int NST = F3 ? ZSTAGES3 : ZSTAGES;
    if (skip && *skip)
        return;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + ZPIPE);
    uint64_t *empty = full + NST;
    uint64_t *done = empty + NST;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *n_issued = abort_flag + 1;
    volatile int *n_consumed = abort_flag + 2;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ti = blockIdx.x / ntj, tj = blockIdx.x - (blockIdx.x / ntj) * ntj;
    const ZSlot sl = slots[blockIdx.y];
    const int np = sl.p1 - sl.p0;
    const int nunits = F3 ? sl.kc1 - sl.kc0 : np * (sl.kc1 - sl.kc0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        *n_issued = 0;
        *n_consumed = 0;
        fence_barrier_init();
    }
    if (warp == 1)
        tmem_alloc(tmem_slot, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            const int ntA = Mpad / ZT, ntB = Npad / ZT;  // 128-row blocks of each operand
            for (int u = 0; u < nunits; ++u) {
                const int s = u % NST;
                const uint32_t ph = (uint32_t)(u / NST) & 1u;
                if (u >= NST && !mbar_wait(&empty[s], ph ^ 1u, wait_ns)) {
                    record_error(err, GW_E_TIMEOUT, SITE_ZGEMM, blockIdx.x);
                    *abort_flag = 1;
                    break;
                }
                if (*abort_flag)
                    break;
                uint8_t *st = smem + s * SB;
                mbar_arrive_expect_tx(&full[s], SB);
                if (F3) {  // A planes 0..3 (hi Re, hi Im, lo Re, lo Im), B planes 0..5 (hi, lo regions)
                    const int kc = sl.kc0 + u;
                    bulk_g2s(st, Ap + ((size_t)kc * ntA + ti) * npA * 2048, 4 * ZPL, &full[s]);
                    bulk_g2s(st + 4 * ZPL, Bp + ((size_t)kc * ntB + tj) * npB * 2048, 4 * ZPL, &full[s]);
                } else {
                    const int kc = sl.kc0 + u / np;  // chunk-major: every pair of a chunk in turn
                    const int2 pr = pairs[sl.p0 + u % np];
                    bulk_g2s(st, Ap + (((size_t)kc * ntA + ti) * npA + 2 * pr.x) * 2048, 2 * ZPL, &full[s]);
                    bulk_g2s(st + 2 * ZPL, Bp + (((size_t)kc * ntB + tj) * npB + 2 * pr.y) * 2048, 2 * ZPL,
                             &full[s]);
                }
                *n_issued = u + 1;
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t ID = mma_idesc(0u, ZT, 2 * ZT, false);  // FP16, N = 256: Re | Im
            constexpr uint32_t ID1 = mma_idesc(0u, ZT, ZT, false), ID1N = mma_idesc(0u, ZT, ZT, true);
            const uint32_t sbase = smem_u32(smem);
            for (int u = 0; u < nunits; ++u) {
                const int s = u % NST;
                if (!mbar_wait(&full[s], (uint32_t)(u / NST) & 1u, wait_ns)) {
                    record_error(err, GW_E_TIMEOUT, SITE_ZGEMM, blockIdx.x);
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t st = sbase + s * SB;
                // Re columns at tmem, Im columns at tmem + ZT
                if (F3) {
                    const uint64_t ahr = smem_desc(st, LBO, SBO), ahi = smem_desc(st + ZPL, LBO, SBO);
                    const uint64_t alr = smem_desc(st + 2 * ZPL, LBO, SBO), ali = smem_desc(st + 3 * ZPL, LBO, SBO);
                    const uint64_t bh_re = smem_desc(st + 4 * ZPL, LBO, SBO), bh_im = smem_desc(st + 5 * ZPL, LBO, SBO);
                    const uint64_t bl_re = smem_desc(st + 6 * ZPL, LBO, SBO), bl_im = smem_desc(st + 7 * ZPL, LBO, SBO);
                    mma_f16(tmem, ahr, bh_re, ID, u > 0 ? 1u : 0u);  // hi * hi
                    mma_f16(tmem, ahi, bh_im, ID1N, 1u);
                    mma_f16(tmem + ZT, ahi, bh_re, ID1, 1u);
                    mma_f16(tmem, ahr, bl_re, ID, 1u);               // hi * lo
                    mma_f16(tmem, ahi, bl_im, ID1N, 1u);
                    mma_f16(tmem + ZT, ahi, bl_re, ID1, 1u);
                    mma_f16(tmem, alr, bh_re, ID, 1u);               // lo * hi
                    mma_f16(tmem, ali, bh_im, ID1N, 1u);
                    mma_f16(tmem + ZT, ali, bh_re, ID1, 1u);
                } else {
                    const uint64_t a_re = smem_desc(st, LBO, SBO), a_im = smem_desc(st + ZPL, LBO, SBO);
                    const uint64_t b_re = smem_desc(st + 2 * ZPL, LBO, SBO);   // rows [Re B; Im B]
                    const uint64_t b_im = smem_desc(st + 3 * ZPL, LBO, SBO);
                    mma_f16(tmem, a_re, b_re, ID, u > 0 ? 1u : 0u);
                    mma_f16(tmem, a_im, b_im, ID1N, 1u);               // -Im A Im B into Re
                    mma_f16(tmem + ZT, a_im, b_re, ID1, 1u);           // Im A Re B into Im
                }
                mma_commit(&empty[s]);
                *n_consumed = u + 1;
            }
            mma_commit(done);  // arrives once every MMA issued above has completed
        }
        __syncwarp();
    } else {
        // epilogue warps 2..5: TMEM lane quarter warp % 4, one output row per thread
        const int q = warp & 3;
        const int row = q * 32 + lane;
        const bool waited = __all_sync(0xffffffffu, mbar_wait(done, 0, wait_ns));
        if (!waited) {
            if (lane == 0)
                record_error(err, GW_E_TIMEOUT, SITE_ZGEMM, blockIdx.x);
            *abort_flag = 1;
        }
        // one decision for the four epilogue warps (the staging below has barriers among them)
        if (!named_bar_or(1, 128, !waited || *abort_flag != 0)) {
            // every copy has landed and every MMA has read it, so the pipeline buffers stage the
            // tile: two halves of 64 columns, each written back as 512-byte row runs
            tc_fence_after();
            const uint32_t base = tmem + ((uint32_t)(q * 32) << 16);
            float2 *stage = reinterpret_cast<float2 *>(smem);  // [128][65]
            const int et = threadIdx.x - 64;                   // 0..127 over the epilogue warps
            for (int h = 0; h < 2; ++h) {
#pragma unroll 1
                for (int c0 = 0; c0 < 64; c0 += 16) {
                    float re[16], im[16];
                    tmem_ld16x2(base + h * 64 + c0, base + ZT + h * 64 + c0, re, im);
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        stage[row * 65 + c0 + i] = make_float2(re[i], im[i]);
                }
                named_bar_sync(1, 128);
                float2 *out = T + ((size_t)blockIdx.y * Mpad + (size_t)ti * ZT) * Npad + (size_t)tj * ZT + h * 64;
                for (int rr = et >> 5; rr < ZT; rr += 4) {
                    const int c = (et & 31) * 2;
                    const float2 a = stage[rr * 65 + c], b2 = stage[rr * 65 + c + 1];
                    *reinterpret_cast<float4 *>(out + (size_t)rr * Npad + c) = make_float4(a.x, a.y, b2.x, b2.y);
                }
                named_bar_sync(1, 128);
            }
        }
        tc_fence_before();
    }

    // ---------------- drain before releasing TMEM and shared memory
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!mbar_wait(done, 0, DRAIN_NS))
            record_error(err, GW_E_TIMEOUT, SITE_ZGEMM, blockIdx.x);
        const int issued = *n_issued, consumed = *n_consumed;
        for (int u = consumed; u < issued; ++u)
            if (!mbar_wait(&full[u % NST], (uint32_t)(u / NST) & 1u, DRAIN_NS)) {
                record_error(err, GW_E_TIMEOUT, SITE_ZGEMM, blockIdx.x);
                break;
            }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 256);
    }
}

// Words of the scalar area (unsigned long long each), zeroed at the start of an inverse.
enum NsWord : int {
    W_EPS = 0,   // max of eps
    W_X,         // max of the current X
    W_XN,        // max of the X being written (moved to W_X by the last block)
    W_Z,         // max of the current Z (2I - eps X) or R
    W_ZN,
    W_DEVN,      // max |out - ref I| being accumulated
    W_RES0,      // residual max |I - eps X| measured by refinement 1 (after phase 1)
    W_RLAST,     // residual measured by the last refinement that ran
    W_NREF,      // refinements that ran
    W_ITERS,     // Newton iterations of phase 1
    W_COUNT,     // completed blocks of the running combine
    W_DISCARD,   // deviations nobody reads
    W_U,         // row-sum bound of lambda_max
    W_UJ,        // the same bound of the Jacobi-scaled matrix
    W_RS2,       // max rs_i^2 (the largest entry of X0 / alpha)
    W_DBAD,      // nonzero: a diagonal entry is not positive and finite (identity start)
    W_TOTAL
};
static_assert(W_TOTAL <= 64, "scalar area");

// What the last block of a combine does with the deviation d = max |out - ref I|.
enum DevUse : int {
    DEV_STORE = 0,   // words[dev_to] = d
    DEV_PHASE1 = 1,  // d < tol: set flags[0] (phase 1 done) and store the iteration count
    DEV_REFINE = 2,  // words[dev_to] = W_RLAST = d, ++W_NREF; d <= tol: set flags[iter + 1 ..]
};

// Block and grid reduction of a combine's two maxima (max(|Re|, |Im|) of out into
// words[acc_max]; deviation into W_DEVN); the last block to finish moves acc_max -> fin_max and
// acts on the deviation as `use` says.
__device__ void combine_tail(float best, float dev, unsigned long long *words, int acc_max, int fin_max, int dev_to,
                             int use, double tol, int iter, int *flags)
{
    __shared__ float red[2][32];
    __shared__ bool last;
    for (int o = 16; o > 0; o >>= 1) {
        best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
        dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    }
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][warp] = best;
        red[1][warp] = dev;
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // one atomic per block and word: same-address atomics serialise
        for (int w = 1; w < nw; ++w) {
            best = fmaxf(best, red[0][w]);
            dev = fmaxf(dev, red[1][w]);
        }
        atomicMax(&words[acc_max], (unsigned long long)__double_as_longlong((double)best));
        atomicMax(&words[W_DEVN], (unsigned long long)__double_as_longlong((double)dev));
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        last = atomicAdd(&words[W_COUNT], 1ull) == (unsigned long long)gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        volatile unsigned long long *vw = words;
        vw[fin_max] = vw[acc_max];
        vw[acc_max] = 0ull;
        const unsigned long long d = vw[W_DEVN];
        const double dv = __longlong_as_double((long long)d);
        vw[W_DEVN] = 0ull;
        vw[W_COUNT] = 0ull;
        if (use == DEV_STORE) {
            vw[dev_to] = d;
        } else if (use == DEV_PHASE1) {
            if (dv < tol) {
                flags[0] = 1;
                vw[W_ITERS] = (unsigned long long)iter;
            }
        } else {
            vw[dev_to] = d;
            vw[W_RLAST] = d;
            vw[W_NREF] = vw[W_NREF] + 1ull;
            if (dv <= tol)
                for (int j = iter + 1; j <= NS_REFINE; ++j)
                    reinterpret_cast<volatile int *>(flags)[j] = 1;
        }
    }
}

__device__ __forceinline__ float finite_or_inf(float d)
{
    return d <= 3.0e38f ? d : __int_as_float(0x7f800000);  // NaN or inf: +inf, which fmaxf keeps
}

// FP16X3 products: out = cI I + cC 2^(eA + eB - 28) sum_slot T[slot] + cD D, the K-range slots
// summed in FP32 (their own rounding is below the split's 2^-22), the rest in FP64.
__global__ void zcombine16_kernel(const float2 *__restrict__ T, int nslots, int Mpad, int Npad,
                                  const unsigned long long *wA, const unsigned long long *wB, int M, int N, double cI,
                                  double cC, const double2 *D, double cD, double2 *out, double ref,
                                  unsigned long long *words, int acc_max, int fin_max, int dev_to, int use, double tol,
                                  int iter, const int *skip, int *flags)
{
    if (skip && *skip)
        return;
    // FP64 runs at 1/64 of the FP32 rate here, so the product part stays in FP32 (it carries the
    // split's 22 bits only) and each entry takes one conversion plus the FP64 terms it needs
    __shared__ float s_sc;
    if (threadIdx.x == 0)
        s_sc = (float)(cC * ldexp(1.0, exp_of(wA) + exp_of(wB) - 28));
    __syncthreads();
    const float sc = s_sc;
    const float cIf = (float)cI, cIref = (float)(cI - ref), cDf = (float)cD;
    float best = 0.f, dev = 0.f;
    const size_t plane = (size_t)Mpad * Npad;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    for (int r = blockIdx.y; r < M && c < N; r += gridDim.y) {
        const size_t i = (size_t)r * N + c;
        const float2 *t = T + (size_t)r * Npad + c;
        float sr = 0.f, si = 0.f;
        for (int s = 0; s < nslots; ++s) {
            const float2 v = t[s * plane];
            sr += v.x;
            si += v.y;
        }
        const float pr = sr * sc, pi = si * sc;  // the product term, exact scaling by 2^k
        double xr = (double)pr, xi = (double)pi;
        float fr = pr, fi = pi, dr = pr;
        if (r == c) {
            xr += cI;
            fr += cIf;
            dr += cIref;
        }
        if (D) {
            const double2 d = D[i];
            xr = fma(cD, d.x, xr);
            xi = fma(cD, d.y, xi);
            fr += cDf * (float)d.x;
            fi += cDf * (float)d.y;
            dr = fr - (r == c ? (float)ref : 0.f);
        }
        out[i] = make_double2(xr, xi);
        best = fmaxf(best, fmaxf(fabsf(fr), fabsf(fi)));
        dev = fmaxf(dev, finite_or_inf(sqrtf(dr * dr + fi * fi)));
    }
    combine_tail(best, dev, words, acc_max, fin_max, dev_to, use, tol, iter, flags);
}

// Exact 128-bit integer -> double (one rounding in each half; the halves do not cancel).
__device__ __forceinline__ double i128_to_double(__int128 a)
{
    const bool neg = a < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)(-a) : (unsigned __int128)a;
    const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
    const double v = hi ? fma((double)hi, 18446744073709551616.0, (double)lo) : (double)lo;
    return neg ? -v : v;
}

// Integer-slice products: every slot tile is an exact integer below 2^24 with weight
// 2^(wexp - 60 + 60) = 2^(-6(d + 2)); sum_slot T 2^(wexp + 60) is added up exactly in 128-bit
// integers, so out = sign (2^(eA + eB - 60) (that sum)) (+ I when identity = 1, added in the same
// integer units, which keeps I - eps X exact) is rounded once.
__global__ void zcombine_int_kernel(const float2 *__restrict__ T, int nslots, const int *__restrict__ wexp, int Mpad,
                                    int Npad, const unsigned long long *wA, const unsigned long long *wB, int M, int N,
                                    int identity, int negate, double2 *out, double ref, unsigned long long *words,
                                    int acc_max, int fin_max, int dev_to, int use, double tol, int iter,
                                    const int *skip, int *flags)
{
    if (skip && *skip)
        return;
    __shared__ int shift[256];
    __shared__ int s_eab;
    __shared__ double s_sc;
    for (int s = threadIdx.x; s < nslots && s < 256; s += blockDim.x)
        shift[s] = wexp[s] + 60;  // 6 (8 - d) in [0, 48]
    if (threadIdx.x == 0) {
        s_eab = exp_of(wA) + exp_of(wB);
        s_sc = ldexp(1.0, s_eab - 60);
    }
    __syncthreads();
    const int eab = s_eab;
    const int ish = 60 - eab;  // I in units of 2^(eab - 60)
    const bool exact_i = ish >= 0 && ish <= 120;
    const double sc = s_sc;
    float best = 0.f, dev = 0.f;
    const size_t plane = (size_t)Mpad * Npad;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    for (int r = blockIdx.y; r < M && c < N; r += gridDim.y) {
        const size_t i = (size_t)r * N + c;
        const float2 *t = T + (size_t)r * Npad + c;
        __int128 ar = 0, ai = 0;
        for (int s = 0; s < nslots; ++s) {
            const float2 v = t[s * plane];
            ar += (__int128)__float2int_rn(v.x) << shift[s];
            ai += (__int128)__float2int_rn(v.y) << shift[s];
        }
        if (negate) {
            ar = -ar;
            ai = -ai;
        }
        const bool diag = identity && r == c;
        if (diag && exact_i)
            ar += (__int128)1 << ish;
        double xr = i128_to_double(ar) * sc, xi = i128_to_double(ai) * sc;
        if (diag && !exact_i)
            xr += 1.0;
        out[i] = make_double2(xr, xi);
        const float fr = (float)xr, fi = (float)xi;
        best = fmaxf(best, fmaxf(fabsf(fr), fabsf(fi)));
        const float dr = r == c ? (float)(xr - ref) : fr;
        dev = fmaxf(dev, finite_or_inf(sqrtf(dr * dr + fi * fi)));
    }
    combine_tail(best, dev, words, acc_max, fin_max, dev_to, use, tol, iter, flags);
}

// rs_i = 1 / sqrt(Re a_ii) (FP32 reciprocal square root, widened) for the Jacobi-scaled start;
// words[W_RS2] = max rs_i^2, words[W_DBAD] set where a diagonal entry gives no positive finite rs.
__global__ void jacobi_rs_kernel(const double2 *__restrict__ A, int n, double *__restrict__ rs,
                                 unsigned long long *words)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double d = A[(size_t)i * n + i].x;
        const double r = (d > 0.0 && d < 1e30) ? (double)rsqrtf((float)d) : 0.0;
        if (r > 0.0 && isfinite(r)) {
            rs[i] = r;
            atomicMax(&words[W_RS2], (unsigned long long)__double_as_longlong(r * r));
        } else {
            rs[i] = 0.0;
            atomicOr(&words[W_DBAD], 1ull);
        }
    }
}

// u = max_i sum_j (|Re a_ij| + |Im a_ij|) >= max_i sum_j |a_ij| >= lambda_max, one warp per row,
// into words[W_U], and the same bound of diag(rs) A diag(rs) into words[W_UJ] (the bits of
// non-negative doubles; zero beforehand).
__global__ void row_sum_bound_kernel(const double2 *__restrict__ A, int n, const double *__restrict__ rs,
                                     unsigned long long *words)
{
    const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int i = blockIdx.x * warps + (threadIdx.x >> 5); i < n; i += gridDim.x * warps) {
        double s = 0.0, sj = 0.0;
        for (int j = lane; j < n; j += 32) {
            const double2 a = A[(size_t)i * n + j];
            const double m = fabs(a.x) + fabs(a.y);
            s += m;
            sj += m * rs[j];
        }
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            sj += __shfl_xor_sync(0xffffffffu, sj, o);
        }
        if (lane == 0) {
            atomicMax(&words[W_U], (unsigned long long)__double_as_longlong(s));
            atomicMax(&words[W_UJ], (unsigned long long)__double_as_longlong(sj * rs[i]));
        }
    }
}

// X0 = c diag(rs)^2 with c = 2 / (1 + u_J) (the Jacobi-scaled start), or c I with c = 2 / (1 + u)
// when words[W_DBAD] is set; both bounds from row_sum_bound_kernel.
__global__ void ns_init_kernel(double2 *X, int N, const double *__restrict__ rs, unsigned long long *words,
                               int *flags)
{
    const bool jac = words[W_DBAD] == 0;
    const double c = 2.0 / (1.0 + __longlong_as_double((long long)words[jac ? W_UJ : W_U]));
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    for (int r = blockIdx.y; r < N && col < N; r += gridDim.y)
        X[(size_t)r * N + col] = make_double2(r == col ? (jac ? c * rs[r] * rs[r] : c) : 0.0, 0.0);
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        const double xmax = jac ? c * __longlong_as_double((long long)words[W_RS2]) : c;
        words[W_X] = (unsigned long long)__double_as_longlong(fabs(xmax));
        words[W_ITERS] = (unsigned long long)NS_MAX;
        for (int j = 0; j <= NS_REFINE + 1; ++j)
            flags[j] = 0;
    }
}

// flags[0]: phase 1 converged.  A failure after a phase 1 that ran out of steps is told apart
// (NS_DETAIL_CAP): the eager form, with more steps, may still converge.
__global__ void ns_final_kernel(const unsigned long long *words, const int *flags, uint32_t *err)
{
    const double r = __longlong_as_double((long long)words[W_RLAST]);
    if (!(r <= NS_ACCEPT))
        record_error(err, GW_E_NUMERIC, SITE_NS, flags[0] ? 0u : NS_DETAIL_CAP);
}

// Grid of the element-wise kernels over an M x N matrix: x covers the columns in 256-thread blocks,
// y strides over the rows, about eight blocks per SM in all.
dim3 grid2d(int M, int N)
{
    const int gx = std::max(1, (N + 255) / 256);
    const int gy = std::max(1, std::min(M, std::max(1, 152 * 8 / gx)));
    return dim3(gx, gy);
}

int round_up(int x, int m)
{
    return ((x + m - 1) / m) * m;
}

}  // namespace

// ---------------------------------------------------------------------------- host side

// Work slots of one product shape: FP16X3 = one slot of the three split pairs per K range (the
// K range split so that tiles x slots fills the GPU); slices = the pairs (t, u) with t + u <= 8,
// grouped by t + u into slots whose exact-sum bound sum 2 m_t m_u K_range stays below 2^24
// (m_0 = 64, m_t = 32) and that hold at most five pairs.
void ZPlan::build(int mode_, int M_, int N_, int K_, int nsm, int slices, int slicesA)
{
    mode = mode_;
    M = M_;
    N = N_;
    K = K_;
    Mpad = round_up(std::max(M, 1), ZT);
    Npad = round_up(std::max(N, 1), ZT);
    nkc = round_up(std::max(K, 1), 16) / 16;
    ntiles = (Mpad / ZT) * (Npad / ZT);
    ns = mode == MODE_FP16X3 ? 2 : std::max(1, std::min(OZ_SLICES, slices > 0 ? slices : OZ_SLICES));
    nsA = std::max(ns, slicesA > 0 ? std::min(OZ_SLICES, slicesA) : ns);  // planes in the A operand
    std::vector<int2> pr;
    std::vector<int> sl, we;  // slot: p0, p1, kc0, kc1
    auto add_slot = [&](int p0, int p1, int kc0, int kc1, int w) {
        sl.insert(sl.end(), {p0, p1, kc0, kc1});
        we.push_back(w);
    };
    if (mode == MODE_FP16X3) {
        pr = {make_int2(0, 0), make_int2(0, 1), make_int2(1, 0)};
        int ks = std::max(1, std::min(std::max(1, nkc / 4), (nsm + ntiles - 1) / ntiles));
        const int per = (nkc + ks - 1) / ks;
        ks = (nkc + per - 1) / per;
        for (int s = 0; s < ks; ++s)
            add_slot(0, 3, s * per, std::min(nkc, (s + 1) * per), -28);
    } else {
        const int ks = (nkc + 127) / 128;  // K range <= 2048: the pair (0, 0) alone stays exact
        const int per = (nkc + ks - 1) / ks;
        const double limit = 16777216.0;
        for (int s = 0; s < ks; ++s) {
            const int kc0 = s * per, kc1 = std::min(nkc, (s + 1) * per);
            const double krange = 16.0 * (kc1 - kc0);
            for (int d = 0; d < ns; ++d) {
                int p0 = static_cast<int>(pr.size());
                double bound = 0.0;
                for (int t = 0; t <= d; ++t) {
                    const int u = d - t;
                    const double b = 2.0 * (t == 0 ? 64 : 32) * (u == 0 ? 64 : 32) * krange;
                    const int cnt = static_cast<int>(pr.size()) - p0;
                    if (cnt > 0 && (bound + b >= limit || cnt == 5)) {
                        add_slot(p0, static_cast<int>(pr.size()), kc0, kc1, -6 * (d + 2));
                        p0 = static_cast<int>(pr.size());
                        bound = 0.0;
                    }
                    pr.push_back(make_int2(t, u));
                    bound += b;
                }
                add_slot(p0, static_cast<int>(pr.size()), kc0, kc1, -6 * (d + 2));
            }
        }
    }
    nslots = static_cast<int>(we.size());
    npairs = static_cast<int>(pr.size());
    host_pairs = pr;
    host_slots = sl;
    host_wexp = we;
}

size_t ZPlan::table_bytes() const
{
    return host_pairs.size() * sizeof(int2) + host_slots.size() * sizeof(int) + host_wexp.size() * sizeof(int);
}

size_t ZPlan::planes_bytes(bool a_operand) const
{
    const int npl = 2;  // Re, Im per slice for both operands
    return (size_t)nkc * (a_operand ? nsA : ns) * npl * (a_operand ? Mpad : Npad) * 16 * sizeof(uint16_t);
}

size_t ZPlan::T_bytes() const
{
    return (size_t)nslots * Mpad * Npad * sizeof(float2);
}

// Copy the slot tables into `tab` (device, table_bytes() long) on stream s.
cudaError_t ZPlan::upload(void *tab, cudaStream_t s)
{
    uint8_t *p = static_cast<uint8_t *>(tab);
    d_pairs = reinterpret_cast<int2 *>(p);
    d_slots = reinterpret_cast<int *>(p + host_pairs.size() * sizeof(int2));
    d_wexp = d_slots + host_slots.size();
    cudaError_t e = cudaMemcpyAsync(d_pairs, host_pairs.data(), host_pairs.size() * sizeof(int2),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_slots, host_slots.data(), host_slots.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_wexp, host_wexp.data(), host_wexp.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    return e;
}

cudaError_t launch_zmaxabs(const double2 *M, int rows, int cols, long ld, unsigned long long *w, cudaStream_t s)
{
    zmaxabs_kernel<<<grid2d(rows, cols), 256, 0, s>>>(M, rows, cols, ld, w);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_zslice(const ZPlan &p, bool a_operand, const double2 *Mx, long ld, const unsigned long long *maxw,
                          uint16_t *planes, const int *skip, cudaStream_t s)
{
    const int rows = a_operand ? p.M : p.N, Rpad = a_operand ? p.Mpad : p.Npad;
    zslice_kernel<<<dim3(p.nkc, Rpad / ZT), 512, 0, s>>>(Mx, ld, rows, p.K, a_operand ? 0 : 1, Rpad, p.mode,
                                                         a_operand ? p.nsA : p.ns,
                                                         2, maxw, planes, skip);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_zgemm16(const ZPlan &p, const uint16_t *Ap, const uint16_t *Bp, float2 *T, uint32_t *err,
                           uint64_t wait_ns, const int *skip, cudaStream_t s)
{
    const bool f3 = p.mode == MODE_FP16X3;
    cudaError_t e = f3 ? cudaFuncSetAttribute(zgemm16_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)ZSMEM)
                       : cudaFuncSetAttribute(zgemm16_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)ZSMEM);
    if (e != cudaSuccess)
        return e;
    dim3 grid(p.ntiles, p.nslots);
    if (f3)
        zgemm16_kernel<true><<<grid, ZTHREADS, ZSMEM, s>>>(Ap, 2 * p.nsA, p.Mpad, Bp, 2 * p.ns, p.Npad, p.d_pairs,
                                                           reinterpret_cast<const ZSlot *>(p.d_slots), p.Npad / ZT,
                                                           T, err, wait_ns, skip);
    else
        zgemm16_kernel<false><<<grid, ZTHREADS, ZSMEM, s>>>(Ap, 2 * p.nsA, p.Mpad, Bp, 2 * p.ns, p.Npad, p.d_pairs,
                                                            reinterpret_cast<const ZSlot *>(p.d_slots), p.Npad / ZT,
                                                            T, err, wait_ns, skip);
    count_launches(1);
    return cudaGetLastError();
}

// out = cI I + cC (A B) + cD D from the slot tiles of plan p.  With integer slices only
// cI in {0, 1}, cC = +-1 and no D are taken (the exact forms the inverse needs).
cudaError_t launch_zcombine(const ZPlan &p, const float2 *T, const unsigned long long *wA,
                            const unsigned long long *wB, double cI, double cC, const double2 *D, double cD,
                            double2 *out, double ref, unsigned long long *words, int acc_max, int fin_max, int dev_to,
                            int use, double tol, int iter, const int *skip, int *flags, cudaStream_t s)
{
    const dim3 grid(grid2d(p.M, p.N));
    if (p.mode == MODE_FP16X3) {
        zcombine16_kernel<<<grid, 256, 0, s>>>(T, p.nslots, p.Mpad, p.Npad, wA, wB, p.M, p.N, cI, cC, D, cD, out, ref,
                                               words, acc_max, fin_max, dev_to, use, tol, iter, skip, flags);
    } else {
        if (D || (cI != 0.0 && cI != 1.0) || (cC != 1.0 && cC != -1.0) || p.nslots > 256)
            return cudaErrorInvalidValue;
        zcombine_int_kernel<<<grid, 256, 0, s>>>(T, p.nslots, p.d_wexp, p.Mpad, p.Npad, wA, wB, p.M, p.N,
                                                 cI == 1.0 ? 1 : 0, cC < 0 ? 1 : 0, out, ref, words, acc_max, fin_max,
                                                 dev_to, use, tol, iter, skip, flags);
    }
    count_launches(1);
    return cudaGetLastError();
}

namespace {
// Carves a workspace into 256-byte aligned pieces; with base == nullptr it only counts.
struct Carver {
    uint8_t *base;
    size_t used = 0;
    explicit Carver(void *b) : base(static_cast<uint8_t *>(b)) {}
    void *take(size_t bytes)
    {
        void *r = base ? base + used : nullptr;
        used += (bytes + 255) / 256 * 256;
        return r;
    }
};

struct GemmWork {
    uint16_t *Ap, *Bp;
    float2 *T;
    unsigned long long *words;
    void *tab;
};

GemmWork carve_gemm(const ZPlan &p, Carver &c)
{
    GemmWork g;
    g.Ap = static_cast<uint16_t *>(c.take(p.planes_bytes(true)));
    g.Bp = static_cast<uint16_t *>(c.take(p.planes_bytes(false)));
    g.T = static_cast<float2 *>(c.take(p.T_bytes()));
    g.words = static_cast<unsigned long long *>(c.take(64 * 8));
    g.tab = c.take(p.table_bytes());
    return g;
}
}  // namespace

// C = A B for M x K and K x N complex128 matrices (row-major, device), by the sliced tensor-core
// product of plan p (mode FP16X3 or integer slices); the workspace holds both operands' planes,
// the slot tiles T, the scalar words and the tables (zgemm_work_bytes).
size_t zgemm_work_bytes(const ZPlan &p)
{
    Carver c(nullptr);
    carve_gemm(p, c);
    return c.used;
}

cudaError_t zgemm_enqueue(ZPlan &p, const double2 *A, long lda, const double2 *B, long ldb, double2 *C, void *work,
                          uint32_t *err, uint64_t wait_ns, cudaStream_t s)
{
    Carver c(work);
    const GemmWork g = carve_gemm(p, c);
    uint16_t *Ap = g.Ap, *Bp = g.Bp;
    float2 *T = g.T;
    unsigned long long *words = g.words;
    cudaError_t e = p.upload(g.tab, s);
    if (e != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(words, 0, 64 * 8, s)) != cudaSuccess)
        return e;
    // words[0], [1]: max of A and B; [2]: max of C (unused), [3]: scratch
    if ((e = launch_zmaxabs(A, p.M, p.K, lda, &words[0], s)) != cudaSuccess)
        return e;
    if ((e = launch_zmaxabs(B, p.K, p.N, ldb, &words[1], s)) != cudaSuccess)
        return e;
    if ((e = launch_zslice(p, true, A, lda, &words[0], Ap, nullptr, s)) != cudaSuccess)
        return e;
    if ((e = launch_zslice(p, false, B, ldb, &words[1], Bp, nullptr, s)) != cudaSuccess)
        return e;
    if ((e = launch_zgemm16(p, Ap, Bp, T, err, wait_ns, nullptr, s)) != cudaSuccess)
        return e;
    // C = 2^(eA + eB) sum_slot 2^wexp T; words[0] and [1] are W_EPS and W_X, untouched here
    return launch_zcombine(p, T, &words[0], &words[1], 0.0, 1.0, nullptr, 0.0, C, 0.0, words, W_ZN, W_Z,
                           W_DISCARD, DEV_STORE, 0.0, 0, nullptr, nullptr, s);
}

namespace {
struct NsWork {
    uint16_t *A16, *AOZ, *XA16, *XB16, *ZB16, *XBOZ;
    float2 *T;
    double2 *X, *Z;
    unsigned long long *words;
    int *skip;
    void *tab16, *taboz, *taboz7;
};

// The first refinement only has to bring max |I - eps X| from the FP16X3 floor (~1e-6) to where
// the second can finish, so its residual uses seven slices (2^-42 relative, 28 slice pairs) of X
// against the nine of eps; the second uses nine (45 pairs).
constexpr int NS_SLICES_FIRST = 7;

void ns_plans(int N, int nsm, ZPlan &p16, ZPlan &poz, ZPlan &poz7)
{
    p16.build(MODE_FP16X3, N, N, N, nsm);
    poz.build(MODE_SLICES, N, N, N, nsm);
    poz7.build(MODE_SLICES, N, N, N, nsm, NS_SLICES_FIRST, OZ_SLICES);
}

NsWork carve_ns(const ZPlan &p16, const ZPlan &poz, const ZPlan &poz7, int N, Carver &c)
{
    NsWork w;
    const size_t nn = (size_t)N * N;
    w.A16 = static_cast<uint16_t *>(c.take(p16.planes_bytes(true)));
    w.AOZ = static_cast<uint16_t *>(c.take(poz.planes_bytes(true)));
    w.XA16 = static_cast<uint16_t *>(c.take(p16.planes_bytes(true)));
    w.XB16 = static_cast<uint16_t *>(c.take(p16.planes_bytes(false)));
    w.ZB16 = static_cast<uint16_t *>(c.take(p16.planes_bytes(false)));
    w.XBOZ = static_cast<uint16_t *>(c.take(poz.planes_bytes(false)));
    w.T = static_cast<float2 *>(c.take(std::max(p16.T_bytes(), std::max(poz.T_bytes(), poz7.T_bytes()))));
    w.X = static_cast<double2 *>(c.take(nn * sizeof(double2)));
    w.Z = static_cast<double2 *>(c.take(nn * sizeof(double2)));
    w.words = static_cast<unsigned long long *>(c.take(64 * 8));
    w.skip = static_cast<int *>(c.take(64));
    w.tab16 = c.take(p16.table_bytes());
    w.taboz = c.take(poz.table_bytes());
    w.taboz7 = c.take(poz7.table_bytes());
    return w;
}
}  // namespace

// eps^-1 by the tensor-core Newton iteration (header comment).  A is eps (N x N, device).
size_t ns_work_bytes(int N, int nsm)
{
    ZPlan p16, poz, poz7;
    ns_plans(N, nsm, p16, poz, poz7);
    Carver c(nullptr);
    carve_ns(p16, poz, poz7, N, c);
    return c.used;
}

// Report of the last inverse run on workspace `work` (synchronous read after the stream is idle):
// out[0] FP16X3 steps of phase 1, [1] residual max |I - eps X| after phase 1, [2] the last measured
// residual, [3] refinements that ran.
cudaError_t ns_report(const void *work, int N, int nsm, double *out4)
{
    ZPlan p16, poz, poz7;
    ns_plans(N, nsm, p16, poz, poz7);
    Carver c(const_cast<void *>(work));
    const NsWork w = carve_ns(p16, poz, poz7, N, c);
    unsigned long long h[W_TOTAL];
    const cudaError_t e = cudaMemcpy(h, w.words, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return e;
    out4[0] = (double)h[W_ITERS];
    out4[1] = __builtin_bit_cast(double, h[W_RES0]);
    out4[2] = __builtin_bit_cast(double, h[W_RLAST]);
    out4[3] = (double)h[W_NREF];
    return cudaSuccess;
}

namespace {
// Host read of a device flag (waits for the stream); a failed read counts as "not set".
bool flag_set(const int *d_flag, cudaStream_t s)
{
    int h = 0;
    if (cudaMemcpyAsync(&h, d_flag, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return h != 0;
}
}  // namespace

// Upload the slot tables of order N into the workspace (done inside ns_inverse_enqueue unless
// the caller did it beforehand, as a captured CUDA graph needs: no pageable copies in capture).
cudaError_t ns_prepare(void *work, int N, int nsm, cudaStream_t s)
{
    ZPlan p16, poz, poz7;
    ns_plans(N, nsm, p16, poz, poz7);
    Carver cv(work);
    const NsWork nw = carve_ns(p16, poz, poz7, N, cv);
    cudaError_t e = p16.upload(nw.tab16, s);
    if (e == cudaSuccess)
        e = poz.upload(nw.taboz, s);
    if (e == cudaSuccess)
        e = poz7.upload(nw.taboz7, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);  // the host tables are locals
    return e;
}

// The kernels of every step check the device flags, so the result does not depend on the host
// reads below: they only stop queuing steps that would return at once (after phase-1 steps 3, 5,
// 7, ... and before the third refinement), at the price of one stream synchronisation each.
// With graph_safe the tables must have been uploaded by ns_prepare and every step is queued (no
// host reads, no pageable copies), so the whole inverse can be captured into a CUDA graph.
cudaError_t ns_inverse_enqueue(const double2 *A, int N, double2 *Xout, void *work, double *rowsum, uint32_t *err,
                               uint64_t wait_ns, int nsm, cudaStream_t s, bool graph_safe, int max_steps)
{
    max_steps = std::max(1, std::min(max_steps, NS_MAX));
    ZPlan p16, poz, poz7;
    ns_plans(N, nsm, p16, poz, poz7);
    Carver cv(work);
    const NsWork nw = carve_ns(p16, poz, poz7, N, cv);
    uint16_t *A16 = nw.A16, *AOZ = nw.AOZ, *XA16 = nw.XA16, *XB16 = nw.XB16, *ZB16 = nw.ZB16, *XBOZ = nw.XBOZ;
    float2 *T = nw.T;
    double2 *X = nw.X, *Z = nw.Z;
    unsigned long long *words = nw.words;
    int *skip = nw.skip;
    void *tab16 = nw.tab16, *taboz = nw.taboz, *taboz7 = nw.taboz7;
    const size_t nn = (size_t)N * N;
    cudaError_t e;
#define NS_TRY(x)                      \
    do {                               \
        if ((e = (x)) != cudaSuccess)  \
            return e;                  \
    } while (0)
    if (graph_safe) {  // the device pointers of the tables, uploaded earlier by ns_prepare
        p16.d_pairs = static_cast<int2 *>(tab16);
        p16.d_slots = reinterpret_cast<int *>(static_cast<uint8_t *>(tab16) + p16.host_pairs.size() * sizeof(int2));
        p16.d_wexp = p16.d_slots + p16.host_slots.size();
        poz.d_pairs = static_cast<int2 *>(taboz);
        poz.d_slots = reinterpret_cast<int *>(static_cast<uint8_t *>(taboz) + poz.host_pairs.size() * sizeof(int2));
        poz.d_wexp = poz.d_slots + poz.host_slots.size();
        poz7.d_pairs = static_cast<int2 *>(taboz7);
        poz7.d_slots =
            reinterpret_cast<int *>(static_cast<uint8_t *>(taboz7) + poz7.host_pairs.size() * sizeof(int2));
        poz7.d_wexp = poz7.d_slots + poz7.host_slots.size();
    } else {
        NS_TRY(p16.upload(tab16, s));
        NS_TRY(poz.upload(taboz, s));
        NS_TRY(poz7.upload(taboz7, s));
    }
    NS_TRY(cudaMemsetAsync(words, 0, 64 * 8, s));
    // eps: its max, both slicings, and the row-sum bound for X0
    NS_TRY(launch_zmaxabs(A, N, N, N, &words[W_EPS], s));
    NS_TRY(launch_zslice(p16, true, A, N, &words[W_EPS], A16, nullptr, s));
    NS_TRY(launch_zslice(poz, true, A, N, &words[W_EPS], AOZ, nullptr, s));
    (void)rowsum;
    double *rs = reinterpret_cast<double *>(Z);  // scratch: Z is first written by phase 1
    jacobi_rs_kernel<<<std::max(1, std::min(152 * 4, (N + 255) / 256)), 256, 0, s>>>(A, N, rs, words);
    row_sum_bound_kernel<<<std::max(1, std::min(152 * 4, (N + 7) / 8)), 256, 0, s>>>(A, N, rs, words);
    count_launches(2);
    ns_init_kernel<<<grid2d(N, N), 256, 0, s>>>(X, N, rs, words, skip);  // skip[0]: phase 1, [1 + j]: refinement j
    count_launches(1);
    NS_TRY(cudaGetLastError());
    // phase 1: X <- X (2I - eps X) with FP16X3 products, stopped on device below NS_TOL
    for (int it = 0; it < max_steps; ++it) {
        NS_TRY(launch_zslice(p16, false, X, N, &words[W_X], XB16, skip, s));
        NS_TRY(launch_zgemm16(p16, A16, XB16, T, err, wait_ns, skip, s));
        // Z = 2I - eps X; deviation |Z - I| = |I - eps X|
        NS_TRY(launch_zcombine(p16, T, &words[W_EPS], &words[W_X], 2.0, -1.0, nullptr, 0.0, Z, 1.0, words, W_ZN, W_Z,
                               W_DISCARD, DEV_PHASE1, NS_TOL, it, skip, skip, s));
        NS_TRY(launch_zslice(p16, true, X, N, &words[W_X], XA16, skip, s));
        NS_TRY(launch_zslice(p16, false, Z, N, &words[W_Z], ZB16, skip, s));
        NS_TRY(launch_zgemm16(p16, XA16, ZB16, T, err, wait_ns, skip, s));
        NS_TRY(launch_zcombine(p16, T, &words[W_X], &words[W_Z], 0.0, 1.0, nullptr, 0.0, X, 0.0, words, W_XN, W_X,
                               W_DISCARD, DEV_STORE, 0.0, it, skip, nullptr, s));
        if (!graph_safe && it >= 3 && (it & 1) && flag_set(skip, s))
            break;
    }
    // phase 2: R = I - eps X to FP64 accuracy (integer slices), X <- X + X R (FP16X3); refinement
    // j runs unless an earlier one measured a residual <= NS_LAST (flag skip[1 + j])
    for (int j = 0; j < NS_REFINE; ++j) {
        const int *sk = skip + 1 + j;
        if (!graph_safe && j == 2 && flag_set(sk, s))
            break;
        const ZPlan &pr = j == 0 ? poz7 : poz;
        NS_TRY(launch_zslice(pr, false, X, N, &words[W_X], XBOZ, sk, s));
        NS_TRY(launch_zslice(p16, true, X, N, &words[W_X], XA16, sk, s));
        NS_TRY(launch_zgemm16(pr, AOZ, XBOZ, T, err, wait_ns, sk, s));
        NS_TRY(launch_zcombine(pr, T, &words[W_EPS], &words[W_X], 1.0, -1.0, nullptr, 0.0, Z, 0.0, words, W_ZN, W_Z,
                               j == 0 ? W_RES0 : W_DISCARD, DEV_REFINE, NS_LAST, j, sk, skip + 1, s));
        NS_TRY(launch_zslice(p16, false, Z, N, &words[W_Z], ZB16, sk, s));
        NS_TRY(launch_zgemm16(p16, XA16, ZB16, T, err, wait_ns, sk, s));
        NS_TRY(launch_zcombine(p16, T, &words[W_X], &words[W_Z], 0.0, 1.0, X, 1.0, X, 0.0, words, W_XN, W_X,
                               W_DISCARD, DEV_STORE, 0.0, j, sk, nullptr, s));
    }
    NS_TRY(cudaMemcpyAsync(Xout, X, nn * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    ns_final_kernel<<<1, 1, 0, s>>>(words, skip, err);
    count_launches(1);
#undef NS_TRY
    return cudaGetLastError();
}

}  // namespace gw
