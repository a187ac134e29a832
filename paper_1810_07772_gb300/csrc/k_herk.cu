// Hermitian rank-k update P(r, r') = -sum_k f_k(r) conj(f_k(r'))  (Eq. Pstatic, written as the
// outer product of the pair densities in Sec. 4.1).  This is the O(N_v N_c N_r^2) term that the
// paper's operation-count table names as dominant.
//
// Tensor-core path (sm_103a, tcgen05):
//   * The complex product is split into real products with A = rows r, B = rows r':
//       Re = Ar Br^T + Ai Bi^T,   Im = Ai Br^T - Ar Bi^T   (the minus via the negate-A bit),
//     accumulated in two FP32 TMEM accumulators of 128 x 256 (all 512 columns).
//   * TF32X3: every FP32 operand is pre-split by the pair-density kernel into hi + lo, both
//     TF32-rounded; each real product is hi*hi + hi*lo + lo*hi (12 MMAs per 8-wide k chunk).
//   * Operands arrive in the canonical no-swizzle K-major layout (8-row x 16-byte core
//     matrices) already in global memory, so each stage is a handful of contiguous 1-D bulk
//     copies (cp.async.bulk) completing on an mbarrier; 4 stages of 48 KB.
//   * One warp lane produces, one lane issues MMAs, and all four warps drain TMEM through
//     shared memory so that the tile and its conjugate mirror are stored with coalesced rows.
//   * Only tiles touching the upper triangle are computed; entries r <= r' are stored directly,
//     entries r > r' as the conjugate mirror (so each element is written exactly once).
#include <cstdlib>
#include <utility>

#include "gw_internal.cuh"
#include "ptx.cuh"

namespace gw {

namespace {

constexpr int BM = HERK_BM, BN = HERK_BN, KC = HERK_KC;
constexpr uint32_t A_BYTES = BM * KC * 4;  // one plane of the A tile: 4 KB
constexpr uint32_t B_BYTES = BN * KC * 4;  // one plane of the B tile: 8 KB
constexpr uint32_t LBO = 128;              // next core matrix along K (4 TF32 further)
constexpr uint32_t SBO = 256;              // next 8-row group
constexpr int EPI_PITCH = 129;             // float2 pitch of the epilogue staging rows
// Limit for the waits that only drain work already in flight after an abort (copies landing,
// MMAs finishing); independent of the caller's wait limit so a tiny limit cannot release
// shared memory or TMEM that is still being written.
constexpr uint64_t DRAIN_NS = 2000000000ull;

template <int SPLIT>
struct HerkCfg {
    static constexpr int NPL = SPLIT == 3 ? 4 : 2;
    static constexpr uint32_t STAGE_BYTES = NPL * (A_BYTES + B_BYTES);
    static constexpr int STAGES = SPLIT == 3 ? 4 : 8;
    static constexpr uint32_t PIPE_BYTES = STAGES * STAGE_BYTES;
    static_assert(PIPE_BYTES >= BM * EPI_PITCH * 8, "epilogue staging must fit in the pipeline buffers");
    static constexpr size_t SMEM = PIPE_BYTES + 256;
};

template <int SPLIT>
__global__ void __launch_bounds__(128, 1)
    herk_tc_kernel(const float *__restrict__ F, int kpad, int nr, int nr_pad, const int2 *__restrict__ tiles,
                   float2 *__restrict__ P, uint32_t *err, uint64_t wait_ns, uint32_t lbo, uint32_t sbo)
{
    using C = HerkCfg<SPLIT>;
    constexpr int NPL = C::NPL;
    constexpr int STAGES = C::STAGES;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + C::PIPE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *tmem_full = empty + STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tmem_full + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *n_issued = abort_flag + 1;
    volatile int *n_consumed = abort_flag + 2;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int2 tile = tiles[blockIdx.x];  // x: 128-row block of r, y: 256-row block of r'
    const int nkc = kpad / KC;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(tmem_full, 1);
        *abort_flag = 0;
        *n_issued = 0;
        *n_consumed = 0;
        fence_barrier_init();
    }
    if (warp == 0)
        tmem_alloc(tmem_slot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t d_re = tmem, d_im = tmem + 256;

    if (warp == 0 && lane == 0) {
        // ---------------- producer: contiguous plane tiles -> shared memory
        const size_t per_chunk = (size_t)nr_pad * KC;
        const size_t a_off = (size_t)tile.x * BM * KC, b_off = (size_t)tile.y * BN * KC;
        for (int kc = 0; kc < nkc; ++kc) {
            const int s = kc % STAGES;
            const uint32_t ph = (kc / STAGES) & 1;
            if (kc >= STAGES && !mbar_wait(&empty[s], ph ^ 1, wait_ns)) {
                record_error(err, GW_E_TIMEOUT, SITE_HERK_PRODUCER, blockIdx.x);
                *abort_flag = 1;
                break;
            }
            if (*abort_flag)
                break;
            uint8_t *st = smem + s * C::STAGE_BYTES;
            mbar_arrive_expect_tx(&full[s], C::STAGE_BYTES);
#pragma unroll
            for (int p = 0; p < NPL; ++p) {
                const float *region = F + ((size_t)kc * NPL + p) * per_chunk;
                bulk_g2s(st + p * A_BYTES, region + a_off, A_BYTES, &full[s]);
                bulk_g2s(st + NPL * A_BYTES + p * B_BYTES, region + b_off, B_BYTES, &full[s]);
            }
            *n_issued = kc + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        constexpr uint32_t ID = mma_idesc(2, BM, BN, false);
        constexpr uint32_t IDN = mma_idesc(2, BM, BN, true);
        const uint32_t sbase = smem_u32(smem);
        for (int kc = 0; kc < nkc; ++kc) {
            const int s = kc % STAGES;
            const uint32_t ph = (kc / STAGES) & 1;
            if (!mbar_wait(&full[s], ph, wait_ns)) {
                record_error(err, GW_E_TIMEOUT, SITE_HERK_MMA, blockIdx.x);
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t st = sbase + s * C::STAGE_BYTES;
            uint64_t a[NPL], b[NPL];
#pragma unroll
            for (int p = 0; p < NPL; ++p) {
                a[p] = smem_desc(st + p * A_BYTES, lbo, sbo);
                b[p] = smem_desc(st + NPL * A_BYTES + p * B_BYTES, lbo, sbo);
            }
            const uint32_t acc = kc > 0 ? 1u : 0u;
            if (SPLIT == 3) {
                // planes: 0 Re hi, 1 Re lo, 2 Im hi, 3 Im lo
                mma_tf32(d_re, a[0], b[0], ID, acc);
                mma_tf32(d_re, a[0], b[1], ID, 1);
                mma_tf32(d_re, a[1], b[0], ID, 1);
                mma_tf32(d_re, a[2], b[2], ID, 1);
                mma_tf32(d_re, a[2], b[3], ID, 1);
                mma_tf32(d_re, a[3], b[2], ID, 1);
                mma_tf32(d_im, a[2], b[0], ID, acc);
                mma_tf32(d_im, a[2], b[1], ID, 1);
                mma_tf32(d_im, a[3], b[0], ID, 1);
                mma_tf32(d_im, a[0], b[2], IDN, 1);
                mma_tf32(d_im, a[0], b[3], IDN, 1);
                mma_tf32(d_im, a[1], b[2], IDN, 1);
            } else {
                // planes: 0 Re, 1 Im
                mma_tf32(d_re, a[0], b[0], ID, acc);
                mma_tf32(d_re, a[1], b[1], ID, 1);
                mma_tf32(d_im, a[1], b[0], ID, acc);
                mma_tf32(d_im, a[0], b[1], IDN, 1);
            }
            mma_commit(&empty[s]);  // frees the stage once these MMAs have read it
            *n_consumed = kc + 1;
        }
        mma_commit(tmem_full);  // arrives when every MMA above has completed (also on abort)
    }
    __syncwarp();

    // ---------------- epilogue: all 128 threads
    const bool ok = __syncthreads_and(mbar_wait(tmem_full, 0, wait_ns) ? 1 : 0) != 0;  // CTA-uniform
    if (!ok) {
        if (threadIdx.x == 0)
            record_error(err, GW_E_TIMEOUT, SITE_HERK_EPILOGUE, blockIdx.x);
        // The MMA lane always commits tmem_full, so this completes once the MMAs already issued
        // have finished; TMEM must not be released before that.
        if (!mbar_wait(tmem_full, 0, DRAIN_NS) && threadIdx.x == 0)
            record_error(err, GW_E_TIMEOUT, SITE_HERK_DRAIN, blockIdx.x);
    }
    const bool write = ok && (*abort_flag == 0) && (nkc > 0);
    __syncthreads();
    tc_fence_after();

    if (write) {
        float2 *stage = reinterpret_cast<float2 *>(smem);  // [128][EPI_PITCH]
        const int m = threadIdx.x;                           // TMEM lane = tile row
        const uint32_t lane_addr = ((uint32_t)(warp * 32) << 16);
        const int r0 = tile.x * BM;
        for (int h = 0; h < 2; ++h) {
            const int c_base = tile.y * BN + h * 128;
            for (int c0 = 0; c0 < 128; c0 += 16) {
                float re[16], im[16];
                tmem_ld16(d_re + lane_addr + h * 128 + c0, re);
                tmem_ld16(d_im + lane_addr + h * 128 + c0, im);
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    stage[m * EPI_PITCH + c0 + q] = make_float2(-re[q], -im[q]);
            }
            __syncthreads();
            // direct rows: P[r][c] for c >= r (real diagonal)
            const int c = c_base + threadIdx.x;
            for (int mm = 0; mm < BM; ++mm) {
                const int r = r0 + mm;
                if (r >= nr)
                    break;
                if (c < nr && c >= r) {
                    float2 v = stage[mm * EPI_PITCH + threadIdx.x];
                    if (c == r)
                        v.y = 0.f;
                    P[(size_t)r * nr + c] = v;
                }
            }
            // mirrored rows: P[c][r] = conj(P[r][c]) for c > r
            const int r = r0 + threadIdx.x;
            for (int cc = 0; cc < 128; ++cc) {
                const int cm = c_base + cc;
                if (cm >= nr)
                    break;
                if (r < nr && r < cm) {
                    const float2 v = stage[threadIdx.x * EPI_PITCH + cc];
                    P[(size_t)cm * nr + r] = make_float2(v.x, -v.y);
                }
            }
            __syncthreads();
        }
    }

    // ---------------- drain: no bulk copy may still target this CTA's shared memory
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int issued = *n_issued, consumed = *n_consumed;
        for (int kc = consumed; kc < issued; ++kc) {
            if (!mbar_wait(&full[kc % STAGES], (kc / STAGES) & 1, DRAIN_NS)) {
                record_error(err, GW_E_TIMEOUT, SITE_HERK_DRAIN, blockIdx.x);
                break;
            }
        }
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ---------------------------------------------------------------------------- CUDA cores
// The same update in plain FP32 FMA: 64 x 64 output tiles, 4 x 4 complex per thread.
constexpr int ST = 64, SK = 16;

__global__ void __launch_bounds__(256)
    herk_simt_kernel(const float2 *__restrict__ F, int kpad, int nr, int nr_pad, float2 *__restrict__ P)
{
    const int bi = blockIdx.y, bj = blockIdx.x;
    if (bj < bi)
        return;  // lower tiles come from the mirror
    __shared__ float2 As[SK][ST];
    __shared__ float2 Bs[SK][ST];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int r0 = bi * ST, c0 = bj * ST;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            acc[i][j] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < kpad; k0 += SK) {
        for (int t = threadIdx.x; t < SK * ST; t += 256) {
            const int kk = t / ST, x = t % ST;
            const int k = k0 + kk;
            As[kk][x] = k < kpad ? F[(size_t)k * nr_pad + r0 + x] : make_float2(0.f, 0.f);
            Bs[kk][x] = k < kpad ? F[(size_t)k * nr_pad + c0 + x] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < SK; ++kk) {
            float2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][ty * 4 + i];
                b[i] = Bs[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // f(r) conj(f(r'))
                    acc[i][j].x = fmaf(a[i].x, b[j].x, fmaf(a[i].y, b[j].y, acc[i][j].x));
                    acc[i][j].y = fmaf(a[i].y, b[j].x, fmaf(-a[i].x, b[j].y, acc[i][j].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty * 4 + i;
        if (r >= nr)
            continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + tx * 4 + j;
            if (c >= nr || c < r)
                continue;
            const float2 v = make_float2(-acc[i][j].x, c == r ? 0.f : -acc[i][j].y);
            P[(size_t)r * nr + c] = v;
            if (c > r)
                P[(size_t)c * nr + r] = make_float2(v.x, -v.y);
        }
    }
}

}  // namespace

size_t herk_smem_bytes(int prec)
{
    return prec == GW_PREC_TF32X1 ? HerkCfg<1>::SMEM : HerkCfg<3>::SMEM;
}

cudaError_t launch_herk_tc(const float *F, int prec, int kpad, int nr, int nr_pad, const int2 *tiles, int n_tiles,
                           float2 *P, uint32_t *err, uint64_t wait_ns, cudaStream_t s)
{
    if (n_tiles <= 0)
        return cudaSuccess;
    const uint32_t lbo = LBO, sbo = SBO;
    cudaError_t e;
    if (prec == GW_PREC_TF32X3) {
        e = cudaFuncSetAttribute(herk_tc_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)HerkCfg<3>::SMEM);
        if (e != cudaSuccess)
            return e;
        herk_tc_kernel<3><<<n_tiles, 128, HerkCfg<3>::SMEM, s>>>(F, kpad, nr, nr_pad, tiles, P, err, wait_ns, lbo, sbo);
        count_launches(1);
    } else {
        e = cudaFuncSetAttribute(herk_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)HerkCfg<1>::SMEM);
        if (e != cudaSuccess)
            return e;
        herk_tc_kernel<1><<<n_tiles, 128, HerkCfg<1>::SMEM, s>>>(F, kpad, nr, nr_pad, tiles, P, err, wait_ns, lbo, sbo);
        count_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_herk_simt(const float2 *F, int kpad, int nr, int nr_pad, float2 *P, cudaStream_t s)
{
    const int nt = nr_pad / ST;
    dim3 grid(nt, nt);
    herk_simt_kernel<<<grid, 256, 0, s>>>(F, kpad, nr, nr_pad, P);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gw
