// Hermitian rank-k update P(r, r') = -sum_k f_k(r) conj(f_k(r')) (Eq. Pstatic; the outer product of
// Sec. 4.1) on 16-bit tensor cores with accumulation accurate to FP32 over very long k.
//
// Why this kernel exists: tcgen05 accumulates in TMEM with FP32 truncation, so the error of one
// long accumulation grows linearly with the number of MMAs into it (about 2e-8 per MMA; 1.7e-4
// at k = 15360).  Here the tensor core only ever accumulates a short window (W chunks of 16 k,
// 9 MMAs per chunk) into a fresh TMEM buffer; eight warps then add the window into FP32
// registers with round-to-nearest, and every L windows the registers are added into the tile's
// own region of P in global memory.  TMEM holds two window buffers so the tensor core keeps
// running while the previous window is promoted.
//
// Operands: every FP32 pair-density value x (scaled by a global power of two s for FP16) is split
// as hi = rn16(x s), lo = rn16(x s - hi); each real product is hi*hi + hi*lo + lo*hi.  FP16 keeps
// 11 significant bits per part (22 together, like the TF32 split) at twice the TF32 MMA rate;
// BF16 keeps 8 + 8.  Complex products: Re = Ar Br^T + Ai Bi^T, Im = Ai Br^T - Ar Bi^T.
//
// The B operand of a chunk sits in shared memory as two adjacent 128-row regions [Bi | Br] per
// hi/lo part, so the 256 rows starting at Bi are [Bi; Br]: one M = 128, N = 256 MMA from A = Ai
// adds Ai Bi^T into the Re columns of the window and Ai Br^T into its Im columns; two N = 128 MMAs
// from A = Ar add Ar Br^T into Re and, with the A-negate bit of the instruction descriptor,
// -Ar Bi^T into Im.  Per chunk that is three N = 256 and six N = 128 MMAs (every output element
// still takes six accumulations), a 32 KB stage of 8 bulk copies and no negated operand copies
// in global memory.  A form with a third region -Bi and six N = 256 MMAs moves fewer bytes through
// shared memory (112 KB per chunk against 116 KB here) but needs 40 KB stages and a fifth and
// sixth plane in global memory; it measured 2-3% slower.
//
// Tiles are 128 x 128, upper triangle only (i <= j); direct and mirrored stores as in the TF32
// kernel, so every element of P is written exactly once at the end.
#include <cuda_bf16.h>
#include <algorithm>
#include <cuda_fp16.h>

#include "gw_internal.cuh"
#include "ptx.cuh"

namespace gw {

namespace {

constexpr int TM = 128, TN = 128, KC16 = HERK16_KC;
constexpr uint32_t PL = TM * KC16 * 2;  // 4 KB: one plane of one 128-row block
// stage: the A block's planes Im hi, Re hi, Im lo, Re lo (4 PL, one bulk copy), then the B
// block's in the same order (one bulk copy): [Im | Re] of the hi part and of the lo part
constexpr uint32_t B_OFF = 4 * PL;
constexpr uint32_t CHUNK_BYTES = 8 * PL;  // 32 KB: one 16-k chunk of A and B
constexpr int PIPE_CHUNKS = 6;            // chunks buffered in shared memory
constexpr uint32_t PIPE_BYTES = PIPE_CHUNKS * CHUNK_BYTES;  // 192 KB
constexpr uint32_t LBO = 128, SBO = 256;
constexpr int EPI_PITCH = 129;
static_assert(PIPE_BYTES >= TM * EPI_PITCH * 8, "epilogue staging must fit");
constexpr size_t SMEM = PIPE_BYTES + 256;
constexpr int NPROMO_WARPS = 8;                  // warps 0..7
constexpr int PRODUCER_WARP = 8, MMA_WARP = 9;
constexpr int NTHREADS = 320;
constexpr uint64_t DRAIN_NS = 2000000000ull;

__device__ __forceinline__ void named_bar(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// CPS: chunks per pipeline stage (1, 2 or 3): fewer, larger stages cost fewer barrier round trips
// per byte; with CPS > 1 every window has its own commit.
template <bool BF16, int CPS>
__global__ void __launch_bounds__(NTHREADS, 1)
    herk16_kernel(const uint16_t *__restrict__ F, int kpad, int nr, int nr_pad, const int2 *__restrict__ tiles,
                  float2 *__restrict__ P, const int *__restrict__ scale_exp, uint32_t *err, uint64_t wait_ns, int W,
                  int L, int split_chunks, long long P_split, int npl)
{
    constexpr int STAGES = PIPE_CHUNKS / CPS;
    constexpr uint32_t STAGE_BYTES = CPS * CHUNK_BYTES;
    static_assert(STAGES * CPS == PIPE_CHUNKS, "stages must tile the pipeline");
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + PIPE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;   // [2] window ready in TMEM buffer b
    uint64_t *acce = accf + 2;         // [2] TMEM buffer b promoted (free)
    uint64_t *done = acce + 2;         // every MMA finished
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *n_issued = abort_flag + 1;
    volatile int *n_consumed = abort_flag + 2;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int2 tile = tiles[blockIdx.x];  // x: 128-row block of r, y: 128-row block of r'
    // split-k: blockIdx.y takes chunks [y split_chunks, (y + 1) split_chunks) and writes its own
    // partial P at P + y P_split (the launcher sizes the splits so that none is empty)
    const int kc_begin = blockIdx.y * split_chunks;
    const int nkc = max(0, min(split_chunks, kpad / KC16 - kc_begin));
    F += (size_t)kc_begin * npl * nr_pad * KC16;  // whole chunks: the same stride in the block layout
    P += (size_t)blockIdx.y * P_split;
    const int nwin = (nkc + W - 1) / W;

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
            // every block's four planes (Im hi, Re hi, Im lo, Re lo) are contiguous: one 16 KB copy
            // for the A rows and one for the B rows per chunk
            const int nblk = nr_pad / TM;
            const int nst = (nkc + CPS - 1) / CPS;
            for (int si = 0; si < nst; ++si) {
                const int s = si % STAGES;
                const uint32_t ph = (si / STAGES) & 1;
                if (si >= STAGES && !mbar_wait(&empty[s], ph ^ 1, wait_ns)) {
                    record_error(err, GW_E_TIMEOUT, SITE_HERK_PRODUCER, blockIdx.x);
                    *abort_flag = 1;
                    break;
                }
                if (*abort_flag)
                    break;
                uint8_t *st = smem + s * STAGE_BYTES;
                const int c0 = si * CPS, nch = min(CPS, nkc - c0);
                mbar_arrive_expect_tx(&full[s], nch * CHUNK_BYTES);
                for (int j = 0; j < nch; ++j) {
                    bulk_g2s(st + j * CHUNK_BYTES, F + plane16_block(c0 + j, tile.x, nblk, npl, 0), 4 * PL, &full[s]);
                    bulk_g2s(st + j * CHUNK_BYTES + B_OFF, F + plane16_block(c0 + j, tile.y, nblk, npl, 0), 4 * PL,
                             &full[s]);
                }
                *n_issued = si + 1;
            }
        }
        __syncwarp();
    } else if (warp == MMA_WARP) {
        if (lane == 0) {
            constexpr uint32_t FMT = BF16 ? 1u : 0u;
            constexpr uint32_t ID = mma_idesc(FMT, TM, 2 * TN, false);  // N = 256: Re | Im columns
            constexpr uint32_t ID1 = mma_idesc(FMT, TM, TN, false), ID1N = mma_idesc(FMT, TM, TN, true);
            const uint32_t sbase = smem_u32(smem);
            int kc = 0;
            bool ok = true;
            for (int win = 0; win < nwin && ok; ++win) {
                const int b = win & 1;
                if (win >= 2 && !mbar_wait(&acce[b], ((win >> 1) - 1) & 1, wait_ns)) {
                    record_error(err, GW_E_TIMEOUT, SITE_HERK_MMA, blockIdx.x);
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + b * 256;  // Re columns d .. d + 127, Im d + 128 .. d + 255
                const int kend = min(nkc, kc + W);
                for (int c = 0; kc < kend; ++kc, ++c) {
                    const int si = kc / CPS, s = si % STAGES;
                    if (kc % CPS == 0 && !mbar_wait(&full[s], (si / STAGES) & 1, wait_ns)) {
                        record_error(err, GW_E_TIMEOUT, SITE_HERK_MMA, blockIdx.x);
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = sbase + s * STAGE_BYTES + (kc % CPS) * CHUNK_BYTES;
                    // both operands staged as Im hi, Re hi, Im lo, Re lo; from Bi the 256 rows are [Bi; Br]
                    const uint64_t a_ih = smem_desc(st, LBO, SBO), a_rh = smem_desc(st + PL, LBO, SBO);
                    const uint64_t a_il = smem_desc(st + 2 * PL, LBO, SBO), a_rl = smem_desc(st + 3 * PL, LBO, SBO);
                    const uint64_t b_ih = smem_desc(st + B_OFF, LBO, SBO), b_rh = smem_desc(st + B_OFF + PL, LBO, SBO);
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
                    if (kc % CPS == CPS - 1 || kc == nkc - 1) {
                        mma_commit(&empty[s]);
                        *n_consumed = si + 1;
                    }
                }
                // With W < STAGES the commit to the empty barrier of the window's last chunk already
                // tells the promotion warps that the window is complete (a commit arrives once every
                // earlier tcgen05 op has finished), and each such commit costs the tensor pipe ~100
                // clocks; a separate window commit is kept only for W >= STAGES (see below).
                if (ok && (CPS > 1 || W >= STAGES))
                    mma_commit(&accf[b]);
            }
            mma_commit(done);  // arrives once every MMA issued above has completed
        }
        __syncwarp();
    } else {
        // ---------------- promotion warps 0..7: TMEM windows -> FP32 registers -> P tile
        const int q = warp & 3;          // TMEM lane quarter
        const int h = warp >> 2;         // column half: 64 h .. 64 h + 63
        const int m = q * 32 + lane;     // tile row
        const int r = tile.x * TM + m;
        const int cbase = tile.y * TN + h * 64;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        float are[64], aim[64];
        int flushed = 0;
        const bool vec_ok = (nr & 1) == 0;  // rows of P start 16-byte aligned
        const int nseg = (nwin + L - 1) / L;
        bool stop = false;
        // Segments of L windows: the registers restart from zero in every segment (a fresh start
        // rather than a conditional reset keeps all 128 sums in registers) and every segment but
        // the last is added into this tile's own region of P.
        for (int seg = 0; seg < nseg && !stop; ++seg) {
#pragma unroll
            for (int i = 0; i < 64; ++i) {
                are[i] = 0.f;
                aim[i] = 0.f;
            }
            const int wend = min(nwin, (seg + 1) * L);
            for (int win = seg * L; win < wend; ++win) {
                const int b = win & 1;
                // Window complete: with W < STAGES the empty barrier of its last chunk; that barrier
                // cannot complete its next phase before this window is promoted (the chunk STAGES later
                // lies in window win + 2 or later, whose MMAs wait for this promotion), so its parity is
                // unambiguous.  With W >= STAGES the window has its own commit on accf[b].
                const int kc_last = min(nkc, (win + 1) * W) - 1;
                const bool own = CPS > 1 || W >= STAGES;  // the window has its own commit
                uint64_t *wbar = own ? &accf[b] : &empty[kc_last % STAGES];
                const uint32_t wpar = own ? (uint32_t)((win >> 1) & 1) : (uint32_t)((kc_last / STAGES) & 1);
                // warp-uniform outcome: the TMEM loads below are warp-collective
                if (!__all_sync(0xffffffffu, mbar_wait(wbar, wpar, wait_ns))) {
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
            // second level: add the registers into this tile's own region of P
            if (r < nr) {
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
        // final sums -> shared staging (the operand pipeline is idle once every window is in)
        named_bar(1, NPROMO_WARPS * 32);
        const bool write = *abort_flag == 0 && nkc > 0;
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
            const int r0 = tile.x * TM, c0 = tile.y * TN;
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

    // ---------------- drain before releasing TMEM and shared memory
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!mbar_wait(done, 0, DRAIN_NS))
            record_error(err, GW_E_TIMEOUT, SITE_HERK_DRAIN, blockIdx.x);
        const int issued = *n_issued, consumed = *n_consumed;  // stages
        for (int si = consumed; si < issued; ++si)
            if (!mbar_wait(&full[si % STAGES], (si / STAGES) & 1, DRAIN_NS)) {
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

int grid_for(size_t n)
{
    size_t g = (n + 255) / 256;
    if (g > 152 * 16)
        g = 152 * 16;
    return g < 1 ? 1 : static_cast<int>(g);
}

}  // namespace

size_t herk16_smem_bytes()
{
    return SMEM;
}

// Sum of the split-k partials of the rank-k update, in a fixed order.
__global__ void sum_parts_kernel(const float2 *__restrict__ parts, int nparts, size_t n, float2 *__restrict__ out)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float2 a = parts[i];
        for (int p = 1; p < nparts; ++p) {
            const float2 b = parts[(size_t)p * n + i];
            a.x += b.x;
            a.y += b.y;
        }
        out[i] = a;
    }
}

template <bool BF16, int CPS>
cudaError_t launch_herk16_t(dim3 grid, cudaStream_t s, const uint16_t *F, int kpad, int nr, int nr_pad,
                            const int2 *tiles, float2 *dst, const int *scale_exp, uint32_t *err, uint64_t wait_ns, int W,
                            int L, int per, long long pstride, int npl)
{
    cudaError_t e = cudaFuncSetAttribute(herk16_kernel<BF16, CPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM);
    if (e != cudaSuccess)
        return e;
    herk16_kernel<BF16, CPS><<<grid, NTHREADS, SMEM, s>>>(F, kpad, nr, nr_pad, tiles, dst, scale_exp, err, wait_ns, W,
                                                          L, per, pstride, npl);
    return cudaSuccess;
}

cudaError_t launch_herk16(const uint16_t *F, bool bf16, int kpad, int nr, int nr_pad, const int2 *tiles, int n_tiles,
                          float2 *P, const int *scale_exp, uint32_t *err, uint64_t wait_ns, int W, int L,
                          cudaStream_t s, int splits, float2 *P_parts, int npl, int cps)
{
    if (n_tiles <= 0)
        return cudaSuccess;
    // Windows of PIPE_CHUNKS or more chunks take their own commit anyway; for them three-chunk
    // stages measured 4 % faster at 24^3 (W = 16: 21.7 against 22.6 ms), for W = 3 within 1 %.
    if (cps == 0)
        cps = W >= PIPE_CHUNKS ? 3 : 1;
    if (cps != 1 && cps != 2 && cps != 3)
        return cudaErrorInvalidValue;
    const int nkc = kpad / KC16;
    if (splits < 1 || !P_parts || nkc < 2)
        splits = 1;
    const int per = (nkc + splits - 1) / splits;
    splits = (nkc + per - 1) / per;  // every split has at least one chunk
    float2 *dst = splits > 1 ? P_parts : P;
    const long long pstride = (long long)nr * nr;
    cudaError_t e;
    dim3 grid(n_tiles, splits);
#define GW_HERK16_LAUNCH(B, C) \
    launch_herk16_t<B, C>(grid, s, F, kpad, nr, nr_pad, tiles, dst, scale_exp, err, wait_ns, W, L, per, pstride, npl)
    if (bf16)
        e = cps == 1 ? GW_HERK16_LAUNCH(true, 1) : cps == 2 ? GW_HERK16_LAUNCH(true, 2) : GW_HERK16_LAUNCH(true, 3);
    else
        e = cps == 1 ? GW_HERK16_LAUNCH(false, 1) : cps == 2 ? GW_HERK16_LAUNCH(false, 2) : GW_HERK16_LAUNCH(false, 3);
#undef GW_HERK16_LAUNCH
    if (e != cudaSuccess)
        return e;
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess || splits == 1)
        return e;
    const size_t n = (size_t)nr * nr;
    sum_parts_kernel<<<grid_for(n), 256, 0, s>>>(P_parts, splits, n, P);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gw
