// Hermitian rank-k update P(r, r') = -sum_k f_k(r) conj(f_k(r')) (Eq. Pstatic; the outer product of
// Sec. 4.1) on CTA pairs: the 2-SM tensor-core operation (tcgen05 cta_group::2) computes one
// 256 x 128 complex tile of P per cluster of two CTAs.
//
// Numerics are those of herk16_kernel: FP16 (or BF16) hi + lo operand planes, three products per
// real product, short TMEM windows of W chunks promoted into FP32 registers, registers added into
// the tile's region of P every L windows.  Each output element takes its 18 accumulations per
// window in the same order as in herk16_kernel.
//
// Why pairs: in the one-CTA kernel every CTA reads its own copy of the B operand from shared
// memory for every MMA, and shared-memory bandwidth (116 KB per 16-k chunk against 768 clocks of
// MMA work) limits it.  In a pair each CTA holds 128 rows of A and HALF of B, so a CTA's shared
// memory moves 80 KB per chunk (32 KB of bulk copies in, 6 x 8 KB read by the MMAs).
//
// Operand split.  A 2-SM MMA with N = 256 takes B columns 0..127 from the even CTA and 128..255
// from the odd one, at the same shared-memory offset.  The Re | Im columns of a window are
//   Re += Ai Bi^T + Ar Br^T,   Im += Ai Br^T - Ar Bi^T,
// so per chunk and hi/lo part the CTAs stage two B regions:
//   region 0 (with A = Ai):  even CTA Bi,  odd CTA Br
//   region 1 (with A = Ar):  even CTA Br,  odd CTA -Bi   (the negated Im planes of F)
// F holds six planes per 128-row block and chunk, Im hi, Im lo, Re hi, Re lo, -Im hi, -Im lo, so
// each CTA fetches its A rows (slots 0..3) and its B regions (even: slots 0..3, odd: 2..5) with
// one 16 KB bulk copy each.
// and the even CTA issues six M = 256, N = 256 MMAs per chunk (Ai x region 0 and Ar x region 1,
// each as hi*hi + hi*lo + lo*hi).
//
// Pipeline and handshakes (every wait bounded by the context's limit; waits on barriers that the
// other CTA or its commits arrive on acquire at cluster scope):
//  * each CTA's producer lane streams its own stage (A planes of its 128 rows, its two B regions)
//    with 1-D bulk copies onto its own `full` barrier;
//  * the odd CTA's relay lane waits for its `full` phase and arrives on the even CTA's `pfull`;
//    the even CTA's MMA lane waits for both before it issues the chunk's MMAs, then commits to the
//    `empty` barrier of BOTH CTAs (multicast), which frees the stage for both producers;
//  * window completion reaches the promotion warps of both CTAs through the same multicast
//    commits; after reading its TMEM each promotion warp arrives on the even CTA's `acce`
//    (16 arrivals: 8 warps per CTA), which lets the MMA lane reuse that TMEM buffer;
//  * at the end the MMA lane commits `done` to both CTAs; each CTA drains its own copies, then
//    both meet at a cluster barrier before TMEM is released and again before exit, so no CTA
//    leaves while its partner may still touch its shared memory or TMEM.
//
// Tiles: pair (I, J) covers rows [256 I, 256 I + 256) and columns [128 J, 128 J + 128), J >= 2 I.
// The odd CTA of a pair with J = 2 I lies below the diagonal and writes nothing.
#include <cuda_bf16.h>
#include <algorithm>
#include <cuda_fp16.h>

#include "gw_internal.cuh"
#include "ptx.cuh"

namespace gw {

namespace {

constexpr int TM = 128, TN = 128, KC16 = HERK16_KC;
constexpr uint32_t PL = TM * KC16 * 2;  // 4 KB: one plane of one 128-row block
// stage: A planes Im hi, Im lo, Re hi, Re lo (4 PL), then B region 0 hi, lo and region 1 hi, lo
constexpr uint32_t B_OFF = 4 * PL;
constexpr uint32_t STAGE_BYTES = 8 * PL;  // 32 KB
constexpr int STAGES = 6;
constexpr uint32_t PIPE_BYTES = STAGES * STAGE_BYTES;  // 192 KB
constexpr uint32_t LBO = 128, SBO = 256;
constexpr int EPI_PITCH = 129;
static_assert(PIPE_BYTES >= TM * EPI_PITCH * 8, "epilogue staging must fit");
constexpr size_t SMEM = PIPE_BYTES + 512;
constexpr int NPROMO_WARPS = 8;                  // warps 0..7
constexpr int PRODUCER_WARP = 8, MMA_WARP = 9;   // warp 9: MMA issuer (even CTA) or relay (odd CTA)
constexpr int NTHREADS = 320;
constexpr uint64_t DRAIN_NS = 2000000000ull;
constexpr int NPL6 = 6;                          // F planes: Re hi, Re lo, Im hi, Im lo, -Im hi, -Im lo

__device__ __forceinline__ void named_bar(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

template <bool BF16>
__global__ void __launch_bounds__(NTHREADS, 1)
    herk16x2_kernel(const uint16_t *__restrict__ F, int kpad, int nr, int nr_pad, const int2 *__restrict__ tiles,
                    float2 *__restrict__ P, const int *__restrict__ scale_exp, uint32_t *err, uint64_t wait_ns,
                    int W, int L)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + PIPE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *pfull = empty + STAGES;  // [STAGES] even CTA: the odd CTA's stage has landed
    uint64_t *accf = pfull + STAGES;   // [2] window ready in TMEM buffer b (W >= STAGES)
    uint64_t *acce = accf + 2;         // [2] even CTA: TMEM buffer b promoted in both CTAs
    uint64_t *done = acce + 2;         // every MMA finished
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *n_issued = abort_flag + 1;
    volatile int *n_consumed = abort_flag + 2;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const int2 tile = tiles[blockIdx.x >> 1];  // x: 256-row block pair, y: 128-column block
    const int ia = 2 * tile.x + (int)rank;     // this CTA's 128-row block of r
    const int nkc = kpad / KC16;
    const int nwin = (nkc + W - 1) / W;
    // the odd CTA of a pair on the diagonal lies below it: it computes but stores nothing
    const bool live = tile.y >= ia;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
            mbar_init(&pfull[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 2 * NPROMO_WARPS);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        *n_issued = 0;
        *n_consumed = 0;
        fence_barrier_init();
    }
    if (warp == MMA_WARP)
        tmem_alloc_pair(tmem_slot, 512);
    tc_fence_before();
    // both CTAs' barriers are initialised and TMEM allocated before anything crosses the pair
    cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == PRODUCER_WARP) {
        if (lane == 0) {
            // six planes per block, Im hi, Im lo, Re hi, Re lo, -Im hi, -Im lo: A is slots 0..3 of this
            // CTA's row block, B slots 0..3 (even CTA: regions Bi, Br) or 2..5 (odd CTA: Br, -Bi) of the
            // column block; one 16 KB bulk copy each
            const int nblk = nr_pad / TM, b_slot = rank == 0 ? P6_IH : P6_RH;
            for (int kc = 0; kc < nkc; ++kc) {
                const int s = kc % STAGES;
                const uint32_t ph = (kc / STAGES) & 1;
                if (kc >= STAGES && !mbar_wait_cluster(&empty[s], ph ^ 1, wait_ns)) {
                    record_error(err, GW_E_TIMEOUT, SITE_HERK_PRODUCER, blockIdx.x);
                    *abort_flag = 1;
                    break;
                }
                if (*abort_flag)
                    break;
                uint8_t *st = smem + s * STAGE_BYTES;
                mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                bulk_g2s(st, F + plane16_block(kc, ia, nblk, NPL6, P6_IH), 4 * PL, &full[s]);
                bulk_g2s(st + B_OFF, F + plane16_block(kc, tile.y, nblk, NPL6, b_slot), 4 * PL, &full[s]);
                *n_issued = kc + 1;
            }
        }
        __syncwarp();
    } else if (warp == MMA_WARP && rank == 1) {
        // relay: tell the even CTA's MMA lane that this CTA's half of the stage has landed
        if (lane == 0) {
            const uint32_t pfull_even = mapa_shared(pfull, 0);
            for (int kc = 0; kc < nkc; ++kc) {
                const int s = kc % STAGES;
                if (!mbar_wait(&full[s], (kc / STAGES) & 1, wait_ns)) {
                    record_error(err, GW_E_TIMEOUT, SITE_HERK_MMA, blockIdx.x);
                    *abort_flag = 1;
                    break;
                }
                *n_consumed = kc + 1;
                mbar_arrive_cluster(pfull_even + 8u * (uint32_t)s);
            }
        }
        __syncwarp();
    } else if (warp == MMA_WARP) {
        if (lane == 0) {
            constexpr uint32_t FMT = BF16 ? 1u : 0u;
            constexpr uint32_t ID = mma_idesc(FMT, 2 * TM, 2 * TN, false);  // M = 256 (pair), N = 256: Re | Im
            const uint32_t sbase = smem_u32(smem);
            int kc = 0;
            bool ok = true;
            for (int win = 0; win < nwin && ok; ++win) {
                const int b = win & 1;
                if (win >= 2 && !mbar_wait_cluster(&acce[b], ((win >> 1) - 1) & 1, wait_ns)) {
                    record_error(err, GW_E_TIMEOUT, SITE_HERK_MMA, blockIdx.x);
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + b * 256;  // Re columns d .. d + 127, Im d + 128 .. d + 255
                const int kend = min(nkc, kc + W);
                for (int c = 0; kc < kend; ++kc, ++c) {
                    const int s = kc % STAGES;
                    const uint32_t par = (kc / STAGES) & 1;
                    if (!mbar_wait(&full[s], par, wait_ns) || !mbar_wait_cluster(&pfull[s], par, wait_ns)) {
                        record_error(err, GW_E_TIMEOUT, SITE_HERK_MMA, blockIdx.x);
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = sbase + s * STAGE_BYTES;
                    // A staged as Im hi, Im lo, Re hi, Re lo; B regions 0 and 1, hi then lo
                    const uint64_t a_ih = smem_desc(st, LBO, SBO), a_il = smem_desc(st + PL, LBO, SBO);
                    const uint64_t a_rh = smem_desc(st + 2 * PL, LBO, SBO), a_rl = smem_desc(st + 3 * PL, LBO, SBO);
                    const uint64_t b0h = smem_desc(st + B_OFF, LBO, SBO), b0l = smem_desc(st + B_OFF + PL, LBO, SBO);
                    const uint64_t b1h = smem_desc(st + B_OFF + 2 * PL, LBO, SBO);
                    const uint64_t b1l = smem_desc(st + B_OFF + 3 * PL, LBO, SBO);
                    const uint32_t acc = c > 0 ? 1u : 0u;
                    mma_f16_pair(d, a_ih, b0h, ID, acc);  // Re += Ai Bi, Im += Ai Br
                    mma_f16_pair(d, a_ih, b0l, ID, 1);
                    mma_f16_pair(d, a_il, b0h, ID, 1);
                    mma_f16_pair(d, a_rh, b1h, ID, 1);    // Re += Ar Br, Im += Ar (-Bi)
                    mma_f16_pair(d, a_rh, b1l, ID, 1);
                    mma_f16_pair(d, a_rl, b1h, ID, 1);
                    mma_commit_pair(&empty[s], 3);
                    *n_consumed = kc + 1;
                }
                // as in herk16_kernel: with W < STAGES the empty commit of the window's last chunk
                // also marks the window complete; a separate window commit only for W >= STAGES
                if (ok && W >= STAGES)
                    mma_commit_pair(&accf[b], 3);
            }
            mma_commit_pair(done, 3);  // arrives in both CTAs once every MMA issued above has completed
        }
        __syncwarp();
    } else {
        // ---------------- promotion warps 0..7: TMEM windows -> FP32 registers -> P tile
        const int q = warp & 3;          // TMEM lane quarter
        const int h = warp >> 2;         // column half: 64 h .. 64 h + 63
        const int m = q * 32 + lane;     // tile row
        const int r = ia * TM + m;
        const int cbase = tile.y * TN + h * 64;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        const uint32_t acce_even = mapa_shared(acce, 0);
        float are[64], aim[64];
        int flushed = 0;
        const bool vec_ok = (nr & 1) == 0;  // rows of P start 16-byte aligned
        const int nseg = (nwin + L - 1) / L;
        bool stop = false;
        for (int seg = 0; seg < nseg && !stop; ++seg) {
#pragma unroll
            for (int i = 0; i < 64; ++i) {
                are[i] = 0.f;
                aim[i] = 0.f;
            }
            const int wend = min(nwin, (seg + 1) * L);
            for (int win = seg * L; win < wend; ++win) {
                const int b = win & 1;
                // window complete: the multicast commit of its last chunk's empty barrier (W <
                // STAGES; the phase argument of herk16_kernel holds, since window win + 2 waits for
                // this promotion in both CTAs) or its own window commit
                const int kc_last = min(nkc, (win + 1) * W) - 1;
                uint64_t *wbar = W < STAGES ? &empty[kc_last % STAGES] : &accf[b];
                const uint32_t wpar = W < STAGES ? (uint32_t)((kc_last / STAGES) & 1) : (uint32_t)((win >> 1) & 1);
                if (!__all_sync(0xffffffffu, mbar_wait_cluster(wbar, wpar, wait_ns))) {
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
                if (lane == 0) {
                    if (rank == 0)
                        mbar_arrive(&acce[b]);
                    else
                        mbar_arrive_cluster(acce_even + 8u * (uint32_t)b);
                }
            }
            if (stop || seg + 1 == nseg)
                break;
            // second level: add the registers into this tile's own region of P
            if (live && r < nr) {
                float2 *row = P + (size_t)r * nr + cbase;
                const int avail = nr - cbase;
                if (vec_ok && avail >= 64) {
                    float4 *r4 = reinterpret_cast<float4 *>(row);
#pragma unroll
                    for (int g = 0; g < 8; ++g) {
                        float4 o[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            o[j] = flushed ? r4[g * 4 + j] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int i = g * 8 + 2 * j;
                            r4[g * 4 + j] = make_float4(o[j].x + are[i], o[j].y + aim[i], o[j].z + are[i + 1],
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
        // final sums -> shared staging.  Every window of this CTA has completed (all MMAs reading
        // this CTA's shared memory are done), so the operand pipeline may be overwritten.
        named_bar(1, NPROMO_WARPS * 32);
        const bool write = *abort_flag == 0 && nkc > 0 && live;
        if (write) {
            const float inv_s2 = ldexpf(1.0f, -2 * (*scale_exp));
            float2 *stage = reinterpret_cast<float2 *>(smem);
            if (flushed && r < nr) {
                const float2 *row = P + (size_t)r * nr + cbase;
                const int avail = nr - cbase;
                if (vec_ok && avail >= 64) {
                    const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
                    for (int g = 0; g < 8; ++g) {
                        float4 o[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            o[j] = r4[g * 4 + j];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int i = g * 8 + 2 * j;
                            are[i] += o[j].x;
                            aim[i] += o[j].y;
                            are[i + 1] += o[j].z;
                            aim[i + 1] += o[j].w;
                        }
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 64; ++i)
                        if (i < avail) {
                            const float2 o = row[i];
                            are[i] += o.x;
                            aim[i] += o.y;
                        }
                }
            }
#pragma unroll
            for (int i = 0; i < 64; ++i)
                stage[m * EPI_PITCH + h * 64 + i] = make_float2(-are[i] * inv_s2, -aim[i] * inv_s2);
        }
        named_bar(1, NPROMO_WARPS * 32);
        if (write) {
            const float2 *stage = reinterpret_cast<const float2 *>(smem);
            const int t = threadIdx.x;  // 0..255
            const int r0 = ia * TM, c0 = tile.y * TN;
            // direct: P[r][c] for c >= r (real diagonal); two rows per pass
            for (int mm = (t >> 7); mm < TM; mm += 2) {
                const int rr = r0 + mm, cc = c0 + (t & 127);
                if (rr < nr && cc < nr && cc >= rr) {
                    float2 v = stage[mm * EPI_PITCH + (t & 127)];
                    if (cc == rr)
                        v.y = 0.f;
                    P[(size_t)rr * nr + cc] = v;
                }
            }
            // mirror: P[c][r] = conj(P[r][c]) for c > r
            for (int cc = (t >> 7); cc < TN; cc += 2) {
                const int cm = c0 + cc, rr = r0 + (t & 127);
                if (cm < nr && rr < nr && rr < cm) {
                    const float2 v = stage[(t & 127) * EPI_PITCH + cc];
                    P[(size_t)cm * nr + rr] = make_float2(v.x, -v.y);
                }
            }
        }
    }

    // ---------------- drain, then release TMEM and leave together
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!mbar_wait_cluster(done, 0, DRAIN_NS))
            record_error(err, GW_E_TIMEOUT, SITE_HERK_DRAIN, blockIdx.x);
        // this CTA's copies that were issued but never waited for (an aborted pipeline)
        const int issued = *n_issued, consumed = *n_consumed;
        for (int kc = consumed; kc < issued; ++kc)
            if (!mbar_wait(&full[kc % STAGES], (kc / STAGES) & 1, DRAIN_NS)) {
                record_error(err, GW_E_TIMEOUT, SITE_HERK_DRAIN, blockIdx.x);
                break;
            }
    }
    tc_fence_before();
    cluster_sync_all();
    if (warp == MMA_WARP) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, 512);
    }
    cluster_sync_all();
}

}  // namespace

size_t herk16x2_smem_bytes()
{
    return SMEM;
}

// Pair tiles (I, J): rows [256 I, 256 I + 256), columns [128 J, 128 J + 128), kept when the pair
// reaches the diagonal (J >= 2 I), in groups of 8 column blocks so that CTAs resident at the same
// time share operand rows in L2.
std::vector<int2> herk_pair_tiles(int nr_pad)
{
    const int npb = nr_pad / (2 * TM), ncb = nr_pad / TN;
    std::vector<int2> t;
    const int GROUP = 8;
    for (int j0 = 0; j0 < ncb; j0 += GROUP)
        for (int I = 0; I < npb; ++I)
            for (int J = j0; J < std::min(ncb, j0 + GROUP); ++J)
                if (J >= 2 * I)
                    t.push_back(make_int2(I, J));
    return t;
}

cudaError_t launch_herk16x2(const uint16_t *F, bool bf16, int kpad, int nr, int nr_pad, const int2 *pair_tiles,
                            int n_pairs, float2 *P, const int *scale_exp, uint32_t *err, uint64_t wait_ns, int W, int L,
                            cudaStream_t s)
{
    if (n_pairs <= 0)
        return cudaSuccess;
    if (nr_pad % (2 * TM) != 0 || kpad % KC16 != 0)
        return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * n_pairs, 1, 1);
    cfg.blockDim = dim3(NTHREADS, 1, 1);
    cfg.dynamicSmemBytes = SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (bf16) {
        e = cudaFuncSetAttribute(herk16x2_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (e == cudaSuccess)
            e = cudaLaunchKernelEx(&cfg, herk16x2_kernel<true>, F, kpad, nr, nr_pad, pair_tiles, P, scale_exp, err,
                                   wait_ns, W, L);
    } else {
        e = cudaFuncSetAttribute(herk16x2_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (e == cudaSuccess)
            e = cudaLaunchKernelEx(&cfg, herk16x2_kernel<false>, F, kpad, nr, nr_pad, pair_tiles, P, scale_exp, err,
                                   wait_ns, W, L);
    }
    if (e != cudaSuccess)
        return e;
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gw
