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
constexpr uint32_t NPL = HERK16_NPL;    // global planes per chunk
// stage: A planes Re hi, Re lo, Im hi, Im lo of the row block (4 PL), then the B regions
// [Im | Re] of the hi part and of the lo part (4 PL)
constexpr uint32_t B_OFF = 4 * PL;
constexpr uint32_t STAGE_BYTES = 8 * PL;  // 32 KB
constexpr int STAGES = 6;
constexpr uint32_t PIPE_BYTES = STAGES * STAGE_BYTES;  // 192 KB
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

template <bool BF16>
__global__ void __launch_bounds__(NTHREADS, 1)
    herk16_kernel(const uint16_t *__restrict__ F, int kpad, int nr, int nr_pad, const int2 *__restrict__ tiles,
                  float2 *__restrict__ P, const int *__restrict__ scale_exp, uint32_t *err, uint64_t wait_ns, int W,
                  int L, int split_chunks, long long P_split)
{
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
    F += (size_t)kc_begin * NPL * nr_pad * KC16;
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
            const size_t per_chunk = (size_t)nr_pad * KC16;  // 16-bit elements per (chunk, plane)
            const size_t a_off = (size_t)tile.x * TM * KC16, b_off = (size_t)tile.y * TN * KC16;
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
                uint8_t *st = smem + s * STAGE_BYTES;
                const uint16_t *chunk = F + (size_t)kc * NPL * per_chunk;
                mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
#pragma unroll
                for (int p = 0; p < 4; ++p)
                    bulk_g2s(st + p * PL, chunk + p * per_chunk + a_off, PL, &full[s]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {  // hi, lo: [Im | Re]
                    uint8_t *bb = st + B_OFF + h * 2 * PL;
                    bulk_g2s(bb, chunk + (2 + h) * per_chunk + b_off, PL, &full[s]);
                    bulk_g2s(bb + PL, chunk + (0 + h) * per_chunk + b_off, PL, &full[s]);
                }
                *n_issued = kc + 1;
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
                    const int s = kc % STAGES;
                    if (!mbar_wait(&full[s], (kc / STAGES) & 1, wait_ns)) {
                        record_error(err, GW_E_TIMEOUT, SITE_HERK_MMA, blockIdx.x);
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = sbase + s * STAGE_BYTES;
                    const uint64_t a_rh = smem_desc(st, LBO, SBO), a_rl = smem_desc(st + PL, LBO, SBO);
                    const uint64_t a_ih = smem_desc(st + 2 * PL, LBO, SBO), a_il = smem_desc(st + 3 * PL, LBO, SBO);
                    // B regions per part: [Bi | Br]; from Bi the 256 rows are [Bi; Br]
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
                    mma_commit(&empty[s]);
                    *n_consumed = kc + 1;
                }
                // With W < STAGES the commit to the empty barrier of the window's last chunk already
                // tells the promotion warps that the window is complete (a commit arrives once every
                // earlier tcgen05 op has finished), and each such commit costs the tensor pipe ~100
                // clocks; a separate window commit is kept only for W >= STAGES (see below).
                if (ok && W >= STAGES)
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
                uint64_t *wbar = W < STAGES ? &empty[kc_last % STAGES] : &accf[b];
                const uint32_t wpar = W < STAGES ? (uint32_t)((kc_last / STAGES) & 1) : (uint32_t)((win >> 1) & 1);
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
        const int issued = *n_issued, consumed = *n_consumed;
        for (int kc = consumed; kc < issued; ++kc)
            if (!mbar_wait(&full[kc % STAGES], (kc / STAGES) & 1, DRAIN_NS)) {
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

// ---------------------------------------------------------------------------- operands
// Bound on max |f| for the FP16 scale: per r, max_v |psi_v(r)| * max_c |psi_c(r)|.
__global__ void f_bound_kernel(const float2 *__restrict__ psiT, int nr, int nb, int nv, unsigned *bound_bits)
{
    // one warp per r: the lanes read the row of psiT coalesced and reduce its two maxima
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    float best = 0.f;
    for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < nr; r += gridDim.x * wpb) {
        float mv = 0.f, mc = 0.f;
        for (int n = lane; n < nb; n += 32) {
            const float2 z = psiT[(size_t)r * nb + n];
            const float a = sqrtf(z.x * z.x + z.y * z.y);
            if (n < nv)
                mv = fmaxf(mv, a);
            else
                mc = fmaxf(mc, a);
        }
        for (int o = 16; o > 0; o >>= 1) {
            mv = fmaxf(mv, __shfl_xor_sync(0xffffffffu, mv, o));
            mc = fmaxf(mc, __shfl_xor_sync(0xffffffffu, mc, o));
        }
        best = fmaxf(best, mv * mc);
    }
    if (lane == 0)
        atomicMax(bound_bits, __float_as_uint(best));  // non-negative floats order like their bits
}

// scale exponent e with (bound * sw_max) * 2^e <= 2^14 (FP16 max is 65504, so a factor of four
// of headroom covers any rounding in the bound); 0 for BF16, which has FP32's exponent range.
__global__ void scale_exp_kernel(const unsigned *bound_bits, float sw_max, int bf16, int *scale_exp)
{
    const float b = __uint_as_float(*bound_bits) * sw_max * 1.001f;
    int e = 0;
    if (!bf16 && b > 0.f && isfinite(b))
        e = (int)floorf(14.0f - log2f(b));
    *scale_exp = max(-100, min(100, e));
}

template <bool BF16>
__device__ __forceinline__ uint16_t to16(float x)
{
    if (BF16) {
        __nv_bfloat16 h = __float2bfloat16_rn(x);
        return *reinterpret_cast<uint16_t *>(&h);
    } else {
        __half h = __float2half_rn(x);
        return *reinterpret_cast<uint16_t *>(&h);
    }
}

template <bool BF16>
__device__ __forceinline__ float from16(uint16_t u)
{
    if (BF16) {
        __nv_bfloat16 h = *reinterpret_cast<__nv_bfloat16 *>(&u);
        return __bfloat162float(h);
    } else {
        __half h = *reinterpret_cast<__half *>(&u);
        return __half2float(h);
    }
}

// The 16-bit operand planes of the pair densities.  blockIdx.y is one 16-wide chunk of k, whose
// (v, c) pairs and weights are resolved once in shared memory; threads run over the chunk in the
// order it is stored (32-bit index arithmetic, no division per element), so every warp writes
// 64 contiguous bytes per plane and reads psi_c(r) for 8 consecutive c of each r.  Used when the
// rows of psiT are too long for pair_density16_rows_kernel.
template <bool BF16>
__global__ void __launch_bounds__(256) pair_density16_kernel(const float2 *__restrict__ psiT,
                                                             const float *__restrict__ sw, int nr, int nb, int nv,
                                                             int nc, int kpad, int nr_pad,
                                                             const int *__restrict__ scale_exp,
                                                             uint16_t *__restrict__ F)
{
    __shared__ int s_v[KC16], s_c[KC16];
    __shared__ float s_w[KC16];
    const int kc = blockIdx.y;
    if (threadIdx.x < KC16) {
        const int k = kc * KC16 + threadIdx.x;
        const float s = ldexpf(1.0f, *scale_exp);
        if (k < nv * nc) {
            const int v = k / nc;
            s_v[threadIdx.x] = v;
            s_c[threadIdx.x] = nv + (k - v * nc);
            s_w[threadIdx.x] = sw[k] * s;
        } else {
            s_v[threadIdx.x] = 0;
            s_c[threadIdx.x] = 0;
            s_w[threadIdx.x] = 0.f;  // padding k: zero operand
        }
    }
    __syncthreads();
    const int per_chunk = nr_pad * KC16;
    uint16_t *Fc = F + (size_t)kc * NPL * per_chunk;
    for (int rem = blockIdx.x * blockDim.x + threadIdx.x; rem < per_chunk; rem += gridDim.x * blockDim.x) {
        const int r = (rem >> 7) * 8 + ((rem & 63) >> 3);  // 8-row group, row in the group
        const int kk = ((rem & 127) >> 6) * 8 + (rem & 7);  // 16-byte core matrix along k, element
        float fr = 0.f, fi = 0.f;
        const float w = s_w[kk];
        if (r < nr && w != 0.f) {
            const float2 a = psiT[(size_t)r * nb + s_v[kk]];
            const float2 b = psiT[(size_t)r * nb + s_c[kk]];
            fr = fmaf(a.x, b.x, a.y * b.y) * w;   // conj(psi_v) psi_c
            fi = fmaf(a.x, b.y, -a.y * b.x) * w;
        }
        const uint16_t rh = to16<BF16>(fr), ih = to16<BF16>(fi), il = to16<BF16>(fi - from16<BF16>(ih));
        Fc[rem] = rh;
        Fc[per_chunk + rem] = to16<BF16>(fr - from16<BF16>(rh));
        Fc[2 * per_chunk + rem] = ih;
        Fc[3 * per_chunk + rem] = il;
    }
}

// The same planes with the rows of psiT staged in shared memory: blockIdx.x is one 8-row group
// (its 8 rows of psiT, nb states each, read from global memory once), blockIdx.y one of
// gridDim.y parts of the k chunks.  Warp w takes chunks w, w + 8, ... of the part; each lane
// makes four consecutive k of one r (the element values are those of pair_density16_kernel, bit
// for bit) and stores 8 bytes per plane, so a warp writes the group's 256 contiguous bytes of
// every plane of a chunk.
constexpr int PD_LDP_PAD = 2;  // row pitch nb + 2 float2: lanes on 8 rows spread over the banks

template <bool BF16>
__global__ void __launch_bounds__(256) pair_density16_rows_kernel(const float2 *__restrict__ psiT,
                                                                  const float *__restrict__ sw, int nr, int nb,
                                                                  int nv, int nc, int kpad, int nr_pad,
                                                                  const int *__restrict__ scale_exp,
                                                                  uint16_t *__restrict__ F)
{
    extern __shared__ __align__(16) uint8_t smem[];
    float2 *s_psi = reinterpret_cast<float2 *>(smem);  // [8][nb + PD_LDP_PAD]
    const int ldp = nb + PD_LDP_PAD;
    const int grp = blockIdx.x;
    for (int t = threadIdx.x; t < 8 * nb; t += blockDim.x) {
        const int rr = t / nb, n = t - rr * nb, r = grp * 8 + rr;
        s_psi[rr * ldp + n] = r < nr ? psiT[(size_t)r * nb + n] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float s = ldexpf(1.0f, *scale_exp);
    const int nk = nv * nc, nchunks = kpad / KC16, per_chunk = nr_pad * KC16;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rem = 4 * lane;                                    // element offset in the group's 128
    const int r8 = (rem & 63) >> 3, kk0 = ((rem & 127) >> 6) * 8 + (rem & 7);
    const bool live = grp * 8 + r8 < nr;
    const float2 *row = s_psi + r8 * ldp;
    const int per_part = (nchunks + gridDim.y - 1) / gridDim.y;
    const int kc_end = min(nchunks, (int)(blockIdx.y + 1) * per_part);
    for (int kc = blockIdx.y * per_part + warp; kc < kc_end; kc += 8) {
        const int k0 = kc * KC16 + kk0;
        int v = k0 / nc, c = k0 - v * nc;
        uint32_t p[4][2];  // planes Re hi, Re lo, Im hi, Im lo: two 16-bit values per word
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = k0 + i;
            float fr = 0.f, fi = 0.f;
            const float w = k < nk ? sw[k] * s : 0.f;  // padding k: zero operand
            if (live && w != 0.f) {
                const float2 a = row[v];
                const float2 b = row[nv + c];
                fr = fmaf(a.x, b.x, a.y * b.y) * w;   // conj(psi_v) psi_c
                fi = fmaf(a.x, b.y, -a.y * b.x) * w;
            }
            if (++c == nc) {
                c = 0;
                ++v;
            }
            const uint16_t rh = to16<BF16>(fr), ih = to16<BF16>(fi), il = to16<BF16>(fi - from16<BF16>(ih));
            const uint32_t h[4] = {rh, to16<BF16>(fr - from16<BF16>(rh)), ih, il};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                p[q][i >> 1] = (i & 1) ? (p[q][i >> 1] | (h[q] << 16)) : h[q];
        }
        uint16_t *dst = F + (size_t)kc * NPL * per_chunk + (size_t)grp * 128 + rem;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint2 *>(dst + (size_t)q * per_chunk) = make_uint2(p[q][0], p[q][1]);
    }
}

// max |M[k][j]| over a complex64 matrix (rows x cols, row stride ld), as float bits.
__global__ void absmax_c64_kernel(const float2 *__restrict__ M, int rows, int cols, long ld, unsigned *bound_bits)
{
    float best = 0.f;
    const size_t total = (size_t)rows * cols;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int k = static_cast<int>(i / cols), j = static_cast<int>(i - (size_t)k * cols);
        const float2 z = M[(size_t)k * ld + j];
        best = fmaxf(best, sqrtf(z.x * z.x + z.y * z.y));
    }
    for (int o = 16; o > 0; o >>= 1)
        best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(bound_bits, __float_as_uint(best));
}

// The 16-bit hi/lo planes of a complex64 matrix M[k][j] (k < rows, j < cols), in the operand
// layout of herk16_kernel with the column index j in the place of r: row k of M is one "pair
// density" of the rank-k update, scaled by 2^scale_exp and split as pair_density16_kernel does.
template <bool BF16>
__global__ void planes16_from_c64_kernel(const float2 *__restrict__ M, int rows, int cols, long ld, int kpad,
                                         int cols_pad, const int *__restrict__ scale_exp, uint16_t *__restrict__ F)
{
    const float s = ldexpf(1.0f, *scale_exp);
    const size_t per_chunk = (size_t)cols_pad * KC16;
    const size_t total = (size_t)(kpad / KC16) * per_chunk;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t kc = i / per_chunk;
        const int rem = static_cast<int>(i - kc * per_chunk);
        const int j = (rem >> 7) * 8 + ((rem & 63) >> 3);
        const int k = static_cast<int>(kc) * KC16 + ((rem & 127) >> 6) * 8 + (rem & 7);
        float fr = 0.f, fi = 0.f;
        if (j < cols && k < rows) {
            const float2 z = M[(size_t)k * ld + j];
            fr = z.x * s;
            fi = z.y * s;
        }
        const uint16_t rh = to16<BF16>(fr), ih = to16<BF16>(fi), il = to16<BF16>(fi - from16<BF16>(ih));
        uint16_t *base = F + kc * NPL * per_chunk + rem;
        base[0] = rh;
        base[per_chunk] = to16<BF16>(fr - from16<BF16>(rh));
        base[2 * per_chunk] = ih;
        base[3 * per_chunk] = il;
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

cudaError_t launch_pair_density16(const float2 *psiT, const float *sw, float sw_max, int nr, int nb, int nv, int nc,
                                  int kpad, int nr_pad, bool bf16, unsigned *bound_bits, int *scale_exp, uint16_t *F,
                                  cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(bound_bits, 0, sizeof(unsigned), s);
    if (e != cudaSuccess)
        return e;
    f_bound_kernel<<<std::max(1, std::min((nr + 7) / 8, 152 * 16)), 256, 0, s>>>(psiT, nr, nb, nv, bound_bits);
    count_launches(1);
    scale_exp_kernel<<<1, 1, 0, s>>>(bound_bits, sw_max, bf16 ? 1 : 0, scale_exp);
    count_launches(1);
    const int nchunks = kpad / KC16, per_chunk = nr_pad * KC16;
    const size_t rows_smem = (size_t)8 * (nb + PD_LDP_PAD) * sizeof(float2);
    if (rows_smem <= 100 * 1024) {
        // parts of k per row group: about 4 blocks per SM-resident slot, at least one chunk per warp
        const int ngrp = nr_pad / 8;
        const int parts = std::max(1, std::min((nchunks + 7) / 8, (152 * 6 * 4 + ngrp - 1) / ngrp));
        const dim3 g2(ngrp, parts);
        e = bf16 ? cudaFuncSetAttribute(pair_density16_rows_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)rows_smem)
                 : cudaFuncSetAttribute(pair_density16_rows_kernel<false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem);
        if (e != cudaSuccess)
            return e;
        if (bf16)
            pair_density16_rows_kernel<true><<<g2, 256, rows_smem, s>>>(psiT, sw, nr, nb, nv, nc, kpad, nr_pad,
                                                                        scale_exp, F);
        else
            pair_density16_rows_kernel<false><<<g2, 256, rows_smem, s>>>(psiT, sw, nr, nb, nv, nc, kpad, nr_pad,
                                                                         scale_exp, F);
        count_launches(1);
        return cudaGetLastError();
    }
    dim3 grid(std::max(1, std::min((per_chunk + 255) / 256, (152 * 16 + nchunks - 1) / nchunks)), nchunks);
    if (bf16)
        pair_density16_kernel<true><<<grid, 256, 0, s>>>(psiT, sw, nr, nb, nv, nc, kpad, nr_pad, scale_exp, F);
    else
        pair_density16_kernel<false><<<grid, 256, 0, s>>>(psiT, sw, nr, nb, nv, nc, kpad, nr_pad, scale_exp, F);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_planes16_from_c64(const float2 *M, int rows, int cols, long ld, int kpad, int cols_pad, bool bf16,
                                     unsigned *bound_bits, int *scale_exp, uint16_t *F, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(bound_bits, 0, sizeof(unsigned), s);
    if (e != cudaSuccess)
        return e;
    absmax_c64_kernel<<<grid_for((size_t)rows * cols), 256, 0, s>>>(M, rows, cols, ld, bound_bits);
    count_launches(1);
    scale_exp_kernel<<<1, 1, 0, s>>>(bound_bits, 1.0f, bf16 ? 1 : 0, scale_exp);
    count_launches(1);
    const size_t total = (size_t)kpad * cols_pad;
    if (bf16)
        planes16_from_c64_kernel<true><<<grid_for(total), 256, 0, s>>>(M, rows, cols, ld, kpad, cols_pad, scale_exp, F);
    else
        planes16_from_c64_kernel<false><<<grid_for(total), 256, 0, s>>>(M, rows, cols, ld, kpad, cols_pad, scale_exp,
                                                                        F);
    count_launches(1);
    return cudaGetLastError();
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

cudaError_t launch_herk16(const uint16_t *F, bool bf16, int kpad, int nr, int nr_pad, const int2 *tiles, int n_tiles,
                          float2 *P, const int *scale_exp, uint32_t *err, uint64_t wait_ns, int W, int L,
                          cudaStream_t s, int splits, float2 *P_parts)
{
    if (n_tiles <= 0)
        return cudaSuccess;
    const int nkc = kpad / KC16;
    if (splits < 1 || !P_parts || nkc < 2)
        splits = 1;
    const int per = (nkc + splits - 1) / splits;
    splits = (nkc + per - 1) / per;  // every split has at least one chunk
    float2 *dst = splits > 1 ? P_parts : P;
    const long long pstride = (long long)nr * nr;
    cudaError_t e;
    dim3 grid(n_tiles, splits);
    if (bf16) {
        e = cudaFuncSetAttribute(herk16_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (e != cudaSuccess)
            return e;
        herk16_kernel<true><<<grid, NTHREADS, SMEM, s>>>(F, kpad, nr, nr_pad, tiles, dst, scale_exp, err, wait_ns, W, L,
                                                         per, pstride);
    } else {
        e = cudaFuncSetAttribute(herk16_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (e != cudaSuccess)
            return e;
        herk16_kernel<false><<<grid, NTHREADS, SMEM, s>>>(F, kpad, nr, nr_pad, tiles, dst, scale_exp, err, wait_ns, W,
                                                          L, per, pstride);
    }
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess || splits == 1)
        return e;
    const size_t n = (size_t)nr * nr;
    sum_parts_kernel<<<grid_for(n), 256, 0, s>>>(P_parts, splits, n, P);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gw
