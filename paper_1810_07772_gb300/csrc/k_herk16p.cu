// Persistent multi-instance variant of the 16-bit Hermitian rank-k update (Eq. Pstatic; the outer
// product of Sec. 4.1) for a batch of independent systems of uneven size.
//
// One CTA per SM walks a static list of (instance, row block, column block) tiles (CTA b takes
// tiles b, b + grid, b + 2 grid, ...; the host orders them by decreasing k so the static schedule
// balances).  The arithmetic per tile is exactly that of herk16_kernel -- the FP16/BF16 hi/lo
// split, W-chunk TMEM windows promoted to FP32 registers, flushes into the tile's region of P
// every L windows -- so every instance's P equals the single-instance result bit for bit.
// What changes is the control: mbarrier phases and the two TMEM window buffers carry across
// tiles, and each tile's final sums go from registers straight to P, so the producer streams the
// next tile's operands while the current tile is being written.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gw_internal.cuh"
#include "ptx.cuh"

namespace gw {

namespace {

constexpr int TM = 128, TN = 128, KC16 = HERK16_KC;
constexpr uint32_t PL = TM * KC16 * 2;  // 4 KB: one plane of one 128-row block
constexpr uint32_t NPL = HERK16_NPL;
// stage as in herk16_kernel: the A block's planes Im hi, Re hi, Im lo, Re lo (one bulk copy), then
// the B block's in the same order, i.e. regions [Im | Re] of the
// hi part and of the lo part, so one N = 256 MMA from A = Im fills the Re and Im columns of a window
constexpr uint32_t B_OFF = 4 * PL;
constexpr uint32_t STAGE_BYTES = 8 * PL;  // 32 KB
constexpr int STAGES = 6;
constexpr uint32_t PIPE_BYTES = STAGES * STAGE_BYTES;
constexpr uint32_t LBO = 128, SBO = 256;
constexpr size_t SMEM = PIPE_BYTES + 256;
constexpr int NPROMO_WARPS = 8;
constexpr int PRODUCER_WARP = 8, MMA_WARP = 9;
constexpr int NTHREADS = 320;
constexpr uint64_t DRAIN_NS = 2000000000ull;

__device__ __forceinline__ void named_bar(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Named barrier that also ORs a predicate over the n participating threads, so a decision to stop
// is the same in every warp (a warp leaving between two named barriers would strand the rest).
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

template <bool BF16>
__global__ void __launch_bounds__(NTHREADS, 1)
    herk16p_kernel(const HerkJob *__restrict__ jobs, const int4 *__restrict__ tiles, int n_tiles, uint32_t *err,
                   uint64_t wait_ns, int W, int L)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + PIPE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;
    uint64_t *acce = accf + 2;
    uint64_t *done = acce + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile long long *n_issued = reinterpret_cast<volatile long long *>(smem + PIPE_BYTES + 192);
    volatile long long *n_consumed = n_issued + 1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], NPROMO_WARPS);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        *n_issued = 0;
        *n_consumed = 0;
        fence_barrier_init();
    }
    if (warp == MMA_WARP)
        tmem_alloc(tmem_slot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == PRODUCER_WARP) {
        if (lane == 0) {
            long long g = 0;  // chunks issued by this CTA over all its tiles
            bool stop = false;
            for (int t = blockIdx.x; t < n_tiles && !stop; t += gridDim.x) {
                const int4 tl = tiles[t];
                const HerkJob jb = jobs[tl.x];
                const int nkc = jb.kpad / KC16;
                const int nblk = jb.nr_pad / TM;  // block layout: one 16 KB copy per operand block
                for (int kc = 0; kc < nkc; ++kc, ++g) {
                    const int s = (int)(g % STAGES);
                    const uint32_t ph = (uint32_t)((g / STAGES) & 1);
                    if (g >= STAGES && !mbar_wait(&empty[s], ph ^ 1, wait_ns)) {
                        record_error(err, GW_E_TIMEOUT, SITE_HERK_PRODUCER, blockIdx.x);
                        *abort_flag = 1;
                        stop = true;
                        break;
                    }
                    if (*abort_flag) {
                        stop = true;
                        break;
                    }
                    uint8_t *st = smem + s * STAGE_BYTES;
                    mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                    bulk_g2s(st, jb.F + plane16_block(kc, tl.y, nblk, NPL, 0), 4 * PL, &full[s]);
                    bulk_g2s(st + B_OFF, jb.F + plane16_block(kc, tl.z, nblk, NPL, 0), 4 * PL, &full[s]);
                    *n_issued = g + 1;
                }
            }
        }
        __syncwarp();
    } else if (warp == MMA_WARP) {
        if (lane == 0) {
            constexpr uint32_t FMT = BF16 ? 1u : 0u;
            constexpr uint32_t ID = mma_idesc(FMT, TM, 2 * TN, false);
            constexpr uint32_t ID1 = mma_idesc(FMT, TM, TN, false), ID1N = mma_idesc(FMT, TM, TN, true);
            const uint32_t sbase = smem_u32(smem);
            long long g = 0, gw = 0;  // chunks and windows consumed by this CTA
            bool ok = true;
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                const int4 tl = tiles[t];
                const int nkc = jobs[tl.x].kpad / KC16;
                const int nwin = (nkc + W - 1) / W;
                int kc = 0;
                for (int win = 0; win < nwin && ok; ++win, ++gw) {
                    const int b = (int)(gw & 1);
                    if (gw >= 2 && !mbar_wait(&acce[b], (uint32_t)(((gw >> 1) - 1) & 1), wait_ns)) {
                        record_error(err, GW_E_TIMEOUT, SITE_HERK_MMA, blockIdx.x);
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + b * 256;
                    const int kend = min(nkc, kc + W);
                    for (int c = 0; kc < kend; ++kc, ++c, ++g) {
                        const int s = (int)(g % STAGES);
                        if (!mbar_wait(&full[s], (uint32_t)((g / STAGES) & 1), wait_ns)) {
                            record_error(err, GW_E_TIMEOUT, SITE_HERK_MMA, blockIdx.x);
                            *abort_flag = 1;
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t st = sbase + s * STAGE_BYTES;
                        const uint64_t a_ih = smem_desc(st, LBO, SBO), a_rh = smem_desc(st + PL, LBO, SBO);
                        const uint64_t a_il = smem_desc(st + 2 * PL, LBO, SBO);
                        const uint64_t a_rl = smem_desc(st + 3 * PL, LBO, SBO);
                        const uint64_t b_ih = smem_desc(st + B_OFF, LBO, SBO);
                        const uint64_t b_rh = smem_desc(st + B_OFF + PL, LBO, SBO);
                        const uint64_t b_il = smem_desc(st + B_OFF + 2 * PL, LBO, SBO);
                        const uint64_t b_rl = smem_desc(st + B_OFF + 3 * PL, LBO, SBO);
                        const uint32_t acc = c > 0 ? 1u : 0u;
                        mma_f16(d, a_ih, b_ih, ID, acc);       // Re += Ai Bi, Im += Ai Br
                        mma_f16(d, a_ih, b_il, ID, 1);
                        mma_f16(d, a_il, b_ih, ID, 1);
                        mma_f16(d, a_rh, b_rh, ID1, 1);        // Re += Ar Br
                        mma_f16(d, a_rh, b_rl, ID1, 1);
                        mma_f16(d, a_rl, b_rh, ID1, 1);
                        mma_f16(d + 128, a_rh, b_ih, ID1N, 1);  // Im -= Ar Bi
                        mma_f16(d + 128, a_rh, b_il, ID1N, 1);
                        mma_f16(d + 128, a_rl, b_ih, ID1N, 1);
                        mma_commit(&empty[s]);
                        *n_consumed = g + 1;
                    }
                    if (ok)
                        mma_commit(&accf[b]);
                }
            }
            mma_commit(done);
        }
        __syncwarp();
    } else {
        // ---------------- promotion warps 0..7
        const int q = warp & 3, h = warp >> 2;
        const int m = q * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        long long gw = 0;
        bool stop = false;
        float are[64], aim[64];
        for (int t = blockIdx.x; t < n_tiles && !stop; t += gridDim.x) {
            const int4 tl = tiles[t];
            const HerkJob jb = jobs[tl.x];
            const int nr = jb.nr;
            float2 *P = jb.P;
            const int r = tl.y * TM + m;
            const int cbase = tl.z * TN + h * 64;
            const int nkc = jb.kpad / KC16;
            const int nwin = (nkc + W - 1) / W;
            const int nseg = (nwin + L - 1) / L;
            const bool vec_ok = (nr & 1) == 0;
            int flushed = 0;
            for (int seg = 0; seg < nseg && !stop; ++seg) {
#pragma unroll
                for (int i = 0; i < 64; ++i) {
                    are[i] = 0.f;
                    aim[i] = 0.f;
                }
                const int wend = min(nwin, (seg + 1) * L);
                for (int win = seg * L; win < wend; ++win, ++gw) {
                    const int b = (int)(gw & 1);
                    if (!__all_sync(0xffffffffu, mbar_wait(&accf[b], (uint32_t)((gw >> 1) & 1), wait_ns))) {
                        if (lane == 0)
                            record_error(err, GW_E_TIMEOUT, SITE_HERK_EPILOGUE, blockIdx.x);
                        *abort_flag = 1;
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = tmem + lane_addr + b * 256 + h * 64;
#pragma unroll
                    for (int c0 = 0; c0 < 64; c0 += 16) {
                        float v[16];
                        tmem_ld16(base + c0, v);
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            are[c0 + i] += v[i];
                        tmem_ld16(base + 128 + c0, v);
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            aim[c0 + i] += v[i];
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0)
                        mbar_arrive(&acce[b]);
                }
                if (stop || seg + 1 == nseg)
                    break;
                if (r < nr) {
                    float2 *row = P + (size_t)r * nr + cbase;
                    const int avail = nr - cbase;
                    if (vec_ok && avail >= 64) {
                        float4 *r4 = reinterpret_cast<float4 *>(row);
#pragma unroll
                        for (int g4 = 0; g4 < 8; ++g4) {
                            float4 o[4];
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                o[j] = flushed ? r4[g4 * 4 + j] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const int i = g4 * 8 + 2 * j;
                                r4[g4 * 4 + j] = make_float4(o[j].x + are[i], o[j].y + aim[i], o[j].z + are[i + 1],
                                                             o[j].w + aim[i + 1]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 64; ++i)
                            if (i < avail) {
                                const float2 o = flushed ? row[i] : make_float2(0.f, 0.f);
                                row[i] = make_float2(o.x + are[i], o.y + aim[i]);
                            }
                    }
                }
                flushed = 1;
            }
            // every promotion warp has finished this tile's flushes before mirrors are written;
            // the stop decision is reduced over all promotion threads so all warps take it
            if (named_bar_or(1, NPROMO_WARPS * 32, stop || *abort_flag != 0))
                break;
            const float s2 = ldexpf(1.0f, -2 * (*jb.scale_exp));
            if (flushed && r < nr) {
                const float2 *row = P + (size_t)r * nr + cbase;
#pragma unroll
                for (int i = 0; i < 64; ++i)
                    if (cbase + i < nr) {
                        const float2 o = row[i];
                        are[i] += o.x;
                        aim[i] += o.y;
                    }
            }
            named_bar(1, NPROMO_WARPS * 32);
            if (r < nr) {
                // direct entries c >= r (real diagonal) from this thread's row
#pragma unroll
                for (int i = 0; i < 64; ++i) {
                    const int col = cbase + i;
                    if (col < nr && col >= r)
                        P[(size_t)r * nr + col] = make_float2(-are[i] * s2, col == r ? 0.f : -aim[i] * s2);
                }
                // mirrored entries P[c][r] = conj(P[r][c]) for c > r (lanes hold consecutive r)
#pragma unroll
                for (int i = 0; i < 64; ++i) {
                    const int col = cbase + i;
                    if (col < nr && col > r)
                        P[(size_t)col * nr + r] = make_float2(-are[i] * s2, aim[i] * s2);
                }
            }
        }
    }

    __syncthreads();
    if (threadIdx.x == 0) {
        if (!mbar_wait(done, 0, DRAIN_NS))
            record_error(err, GW_E_TIMEOUT, SITE_HERK_DRAIN, blockIdx.x);
        const long long issued = *n_issued, consumed = *n_consumed;
        for (long long g = consumed; g < issued; ++g)
            if (!mbar_wait(&full[g % STAGES], (uint32_t)((g / STAGES) & 1), DRAIN_NS)) {
                record_error(err, GW_E_TIMEOUT, SITE_HERK_DRAIN, blockIdx.x);
                break;
            }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == MMA_WARP) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

}  // namespace

cudaError_t launch_herk16p(const HerkJob *jobs, const int4 *tiles, int n_tiles, int grid, bool bf16, uint32_t *err,
                           uint64_t wait_ns, int W, int L, cudaStream_t s)
{
    if (n_tiles <= 0)
        return cudaSuccess;
    cudaError_t e;
    if (bf16) {
        e = cudaFuncSetAttribute(herk16p_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (e != cudaSuccess)
            return e;
        herk16p_kernel<true><<<grid, NTHREADS, SMEM, s>>>(jobs, tiles, n_tiles, err, wait_ns, W, L);
    } else {
        e = cudaFuncSetAttribute(herk16p_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (e != cudaSuccess)
            return e;
        herk16p_kernel<false><<<grid, NTHREADS, SMEM, s>>>(jobs, tiles, n_tiles, err, wait_ns, W, L);
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gw
