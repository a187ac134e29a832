// Tensor-core inference of the correction network (n_in -> 256 -> 256 -> 256 -> 2, tanh), one
// persistent kernel on CTA pairs (tcgen05 cta_group::2).
//
// A pair takes 256 input rows at a time, 128 per CTA.  Each 2-SM MMA has M = 256 (the pair's
// rows; each CTA supplies its 128 from its own shared memory) and N = 256 (the 256 outputs of a
// layer; the even CTA supplies the B rows of outputs 0..127, the odd CTA those of 128..255), and
// each CTA's TMEM receives its 128 rows x 256 outputs.  So a CTA holds HALF of every weight matrix,
// and all three stay resident: W1 | W1 (8 KB), W2 (64 KB), W3 (64 KB), plus the 64 KB operand A.
//
// Per 256-row tile, three MMA phases into two alternating 256-column TMEM regions:
//   layer 1: A = [x_hi | x_lo] (the FP32 inputs split into two FP16 parts, K = 32 with n_in <= 16
//            per part), B = [W1 | W1]: x W1^T to FP32 accuracy in two MMAs;
//   layer 2: A = h1 (FP16), B = W2, 16 MMAs of K = 16;
//   layer 3: A = h2 (FP16), B = W3.
// Epilogue warps (16: TMEM lane quarter x 64-column quarter) read a finished layer from TMEM, add
// the bias, take tanh and write the FP16 result into A as the next layer's operand.  Each warp
// writes its four K chunks in turn; round j (chunk j of every warp, K chunks 4 g + j) is signalled
// on a CTA-local barrier, which one relay lane of the odd CTA forwards to the even CTA, so the next
// layer's MMAs trail the epilogue by one round.  Layer 3's epilogue applies the 256 -> 2 output
// layer in FP32 and sums the four column quarters in a fixed order.  The next tile's inputs go into
// A (chunks 0 and 1) as soon as layer 3's MMAs are done, so its layer 1 overlaps that epilogue.
//
// tanh: tanh.approx.f32 (hardware, relative error about 2^-11).  h1 and h2 are rounded to FP16
// after it (FP16 operands of the next product); h3 stays FP32.
//
// Every wait is bounded (the caller's limit); a CTA that gives up records GW_E_TIMEOUT and stops.
// No thread of the loop waits on a barrier without a limit: the cross-warp hand-offs inside the
// loop are mbarriers, and the CTAs meet at cluster barriers only before the loop and after every
// warp has left it.  Operand layout (K-major, no swizzle): 16-wide K chunks of 8-row x 16-byte core
// matrices, 128 bytes apart along K and 256 bytes apart along M / N.
#include <algorithm>
#include <cuda_fp16.h>

#include "gw_internal.cuh"
#include "ptx.cuh"

namespace gw {

namespace {

constexpr int TCH = 256;                      // hidden width of the tensor-core path
constexpr int TROWS = 128;                    // rows per CTA, 256 per pair
constexpr int MAX_IN = 16;                    // inputs of layer 1 on this path
constexpr uint32_t CH = TROWS * 16 * 2;       // 4 KB: one K chunk of 128 rows (A) or 128 outputs (B half)
constexpr uint32_t A_BYTES = 16 * CH;         // 64 KB
constexpr uint32_t W1H = 2 * CH;              // 8 KB: half of layer 1's B (W1 | W1, K = 32)
constexpr uint32_t WH = 16 * CH;              // 64 KB: half of W2 or W3
constexpr uint32_t WT_BYTES = 2 * W1H + 4 * WH;  // the tiled weights of both halves
constexpr uint32_t OFF_W2 = W1H, OFF_W3 = OFF_W2 + WH, OFF_A = OFF_W3 + WH, OFF_F = OFF_A + A_BYTES;
constexpr int NFLT = 3 * TCH + 2 * TCH + 4;   // b1 | b2 | b3, W4 [2][256], b4
constexpr uint32_t OFF_PART = OFF_F + NFLT * 4;                // float2 [2][4][128]
constexpr uint32_t OFF_BAR = OFF_PART + 2 * 4 * TROWS * 8;
enum { B_W = 0, B_WPEER = 1, B_RDY = 2, B_RRDY = 6, B_ACC = 10, B_Y = 13, B_DONE = 14, NBARS = 15 };
constexpr size_t SMEM = OFF_BAR + NBARS * 8 + 16;
constexpr int NEPI = 16;                      // epilogue warps 0..15
constexpr int CTRL_WARP = 16;                 // weights, MMA issue (even CTA), weight relay (odd CTA)
constexpr int NTHREADS = (NEPI + 1) * 32;
constexpr uint32_t IDESC = mma_idesc(0, 2 * TROWS, TCH, false);  // M = 256 (pair), N = 256
constexpr uint64_t DRAIN_NS = 2000000000ull;
static_assert(OFF_PART % 8 == 0 && OFF_BAR % 8 == 0, "alignment");
static_assert(SMEM <= 232448, "shared memory per CTA");

__host__ __device__ constexpr uint32_t a_off(int m, int k)
{
    return (k >> 4) * CH + (m >> 3) * 256 + ((k >> 3) & 1) * 128 + (m & 7) * 16 + (k & 7) * 2;
}

// Output n (0..255) and input k of a weight matrix with nk K chunks, split into the two CTAs' halves.
__host__ __device__ constexpr uint32_t w_off(int n, int k, int nk)
{
    return (n >> 7) * (nk * CH) + a_off(n & 127, k);
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ float tanh_fast(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// A warp's TMEM load of 32 lanes x 16 columns, issued without waiting: r is valid only after
// tmem_wait(r).
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

// Wait for this thread's TMEM loads.  The registers of the load being waited for pass through the
// statement, so that no use of them is scheduled before it.
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// Two FP32 values rounded to FP16 (round to nearest even) in one packed conversion, a in the low half.
__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Row-major FP16 weights (out x in) -> the halves' operand layout: W1 (256 x n_in) twice along K
// (K = 32, zero beyond n_in in each copy), then W2 and W3 (256 x 256).
__global__ void tile_weights_kernel(const __half *__restrict__ W1, int n_in, const __half *__restrict__ W2,
                                    const __half *__restrict__ W3, uint8_t *__restrict__ Wt)
{
    constexpr int N1 = TCH * 32, N2 = TCH * TCH;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N1 + 2 * N2; t += gridDim.x * blockDim.x) {
        if (t < N1) {
            const int n = t >> 5, k = t & 31, kk = k & 15;
            const __half v = kk < n_in ? W1[n * n_in + kk] : __float2half_rn(0.f);
            *reinterpret_cast<__half *>(Wt + w_off(n, k, 2)) = v;
        } else {
            const int u = t - N1, mtx = u / N2, e = u - mtx * N2, n = e / TCH, k = e - n * TCH;
            *reinterpret_cast<__half *>(Wt + 2 * W1H + mtx * 2 * WH + w_off(n, k, 16)) = (mtx ? W3 : W2)[e];
        }
    }
}

__global__ void __launch_bounds__(NTHREADS, 1)
    mlp_tc_pair_kernel(const float *__restrict__ X, long n, int n_in, const uint8_t *__restrict__ Wt,
                       const float *__restrict__ b1, const float *__restrict__ b2, const float *__restrict__ b3,
                       const __half *__restrict__ W4, const float *__restrict__ b4, float *__restrict__ Y,
                       uint32_t *err, uint64_t wait_ns)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sA = smem + OFF_A;
    float *sb = reinterpret_cast<float *>(smem + OFF_F);  // b1 [0, 256), b2 [256, 512), b3 [512, 768)
    float *sW4 = sb + 3 * TCH;                             // [2][256]
    float *sb4 = sW4 + 2 * TCH;
    float2 *part = reinterpret_cast<float2 *>(smem + OFF_PART);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + OFF_BAR);
    uint64_t *rdy = bars + B_RDY;      // [4] round j of A (chunks 4 g + j) written in this CTA
    uint64_t *rrdy = bars + B_RRDY;    // [4] even CTA: ... and in the odd CTA (relayed)
    uint64_t *accfull = bars + B_ACC;  // [3] layer l's products of the current tile are in TMEM
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + NBARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    volatile int *w_landed = abort_flag + 1;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t rank = cluster_ctarank();
    const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
    const int ntiles = (int)((n + 2 * TROWS - 1) / (2 * TROWS));

    if (tid == 0) {
        mbar_init(&bars[B_W], 1);
        mbar_init(&bars[B_WPEER], 1);
        for (int j = 0; j < 4; ++j) {
            mbar_init(&rdy[j], NEPI);
            mbar_init(&rrdy[j], 1);
        }
        for (int l = 0; l < 3; ++l)
            mbar_init(&accfull[l], 1);
        mbar_init(&bars[B_Y], NEPI);
        mbar_init(&bars[B_DONE], 1);
        *abort_flag = 0;
        *w_landed = 0;
        fence_barrier_init();
    }
    if (warp == CTRL_WARP)
        tmem_alloc_pair(tslot, 512);
    for (int t = tid; t < TCH; t += NTHREADS) {
        sb[t] = b1[t];
        sb[TCH + t] = b2[t];
        sb[2 * TCH + t] = b3[t];
        sW4[t] = __half2float(W4[t]);
        sW4[TCH + t] = __half2float(W4[TCH + t]);
    }
    if (tid < 2)
        sb4[tid] = b4[tid];
    tc_fence_before();
    // both CTAs' barriers are initialised and TMEM allocated before anything crosses the pair
    cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == CTRL_WARP) {
        // The whole warp runs this loop (every lane polls the barriers, so the warp stays converged);
        // lane 0 alone issues copies, MMAs and commits.
        const bool leader = lane == 0;
        if (leader) {
            mbar_arrive_expect_tx(&bars[B_W], W1H + 2 * WH);
            bulk_g2s(smem, Wt + rank * W1H, W1H, &bars[B_W]);
            bulk_g2s(smem + OFF_W2, Wt + 2 * W1H + rank * WH, WH, &bars[B_W]);
            bulk_g2s(smem + OFF_W3, Wt + 2 * W1H + 2 * WH + rank * WH, WH, &bars[B_W]);
        }
        bool ok = __all_sync(0xffffffffu, mbar_wait(&bars[B_W], 0, wait_ns));
        if (ok && leader)
            *w_landed = 1;
        if (rank == 1) {
            if (ok && leader)
                mbar_arrive_cluster(mapa_shared(&bars[B_WPEER], 0));
            // Relay: each round of this CTA's A, once its 16 epilogue warps have arrived on the local
            // barrier, goes to the even CTA's MMA lane as one arrival at cluster scope (the warps'
            // own arrivals stay CTA-local: sixteen cluster-scope releases per chunk serialise).  The
            // rounds come in the order the MMA lane consumes them.
            const uint32_t rrdy_even = mapa_shared(rrdy, 0);
            auto relay = [&](int j, uint32_t par) {
                if (!__all_sync(0xffffffffu, mbar_wait(&rdy[j], par, wait_ns)))
                    return false;
                if (leader)
                    mbar_arrive_cluster(rrdy_even + 8u * (uint32_t)j);
                __syncwarp();
                return true;
            };
            for (int t = pair, i = 0; ok && t < ntiles; t += npairs, ++i) {
                if (*abort_flag)
                    break;
                ok = relay(0, (3 * i) & 1);
                for (int l = 1; l <= 2 && ok; ++l)
                    for (int j = 0; j < 4 && ok; ++j)
                        ok = relay(j, j == 0 ? (3 * i + l) & 1 : (2 * i + l - 1) & 1);
            }
        } else {
            ok = ok && __all_sync(0xffffffffu, mbar_wait_cluster(&bars[B_WPEER], 0, wait_ns));
            // round j of A is ready in both CTAs
            auto wait_round = [&](int j, uint32_t par) {
                return __all_sync(0xffffffffu,
                                  mbar_wait(&rdy[j], par, wait_ns) && mbar_wait_cluster(&rrdy[j], par, wait_ns));
            };
            // Descriptors are built once; chunk c is c * CH bytes further, c * CH / 16 in the address
            // field (every operand lies below 256 KB, so the field does not overflow).  The issue loop
            // is kept short: one MMA per ~130 clocks of tensor work needs the lane to issue that fast.
            const uint32_t sbase = smem_u32(smem);
            const uint64_t a0 = smem_desc(smem_u32(sA), 128, 256), w1 = smem_desc(sbase, 128, 256);
            const uint64_t w2 = smem_desc(sbase + OFF_W2, 128, 256), w3 = smem_desc(sbase + OFF_W3, 128, 256);
            constexpr uint64_t CHD = CH >> 4;
            for (int t = pair, i = 0; ok && t < ntiles; t += npairs, ++i) {
                if (*abort_flag)
                    break;
                // layer 1: the inputs' two FP16 parts against W1 twice
                if (!wait_round(0, (3 * i) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                uint32_t d = tmem + ((3 * i) & 1) * 256;
                if (leader) {
                    mma_f16_pair(d, a0, w1, IDESC, 0);
                    mma_f16_pair(d, a0 + CHD, w1 + CHD, IDESC, 1);
                    mma_commit_pair(&accfull[0], 3);
                }
                __syncwarp();
                for (int l = 1; l <= 2 && ok; ++l) {
                    d = tmem + ((3 * i + l) & 1) * 256;
                    const uint64_t b0 = l == 1 ? w2 : w3;
                    const uint32_t par0 = (3 * i + l) & 1, par = (2 * i + l - 1) & 1;
                    // rounds j of four chunks 4 g + j, one from each column quarter of the epilogue,
                    // which finish together
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        ok = wait_round(j, j == 0 ? par0 : par);
                        if (!ok)
                            break;
                        tc_fence_after();
                        if (leader) {
#pragma unroll
                            for (int g = 0; g < 4; ++g) {
                                const int c = 4 * g + j;
                                mma_f16_pair(d, a0 + c * CHD, b0 + c * CHD, IDESC, (j | g) ? 1u : 0u);
                            }
                        }
                        __syncwarp();
                    }
                    if (ok && leader)
                        mma_commit_pair(&accfull[l], 3);
                    __syncwarp();
                }
            }
            // arrives in both CTAs once every MMA issued above has completed
            if (leader)
                mma_commit_pair(&bars[B_DONE], 3);
            __syncwarp();
        }
        if (!ok && leader) {
            record_error(err, GW_E_TIMEOUT, SITE_HERK_MMA, blockIdx.x);
            *abort_flag = 1;
        }
        __syncwarp();
    } else {
        // ---------------- epilogue warps: TMEM lane quarter q, columns 64 cq .. 64 cq + 63
        const int q = warp & 3, cq = warp >> 2, m = q * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        auto signal = [&](int j) {
            fence_proxy_async_smem();  // the tensor core reads what this warp just wrote
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&rdy[j]);
        };
        // the inputs of tile t, split into FP16 hi and lo parts, as K chunks 0 and 1 of A
        auto write_x = [&](int t) {
            const long row = (long)t * 2 * TROWS + rank * TROWS + m;
            float x[MAX_IN];
#pragma unroll
            for (int k = 0; k < MAX_IN; ++k)
                x[k] = (k < n_in && row < n) ? X[row * n_in + k] : 0.f;
            uint32_t hi[8], lo[8];
#pragma unroll
            for (int k = 0; k < MAX_IN; k += 2) {
                const __half2 h = __floats2half2_rn(x[k], x[k + 1]);
                hi[k >> 1] = *reinterpret_cast<const uint32_t *>(&h);
                lo[k >> 1] = pack2(x[k] - __low2float(h), x[k + 1] - __high2float(h));
            }
            *reinterpret_cast<uint4 *>(sA + a_off(m, 0)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(sA + a_off(m, 8)) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
            *reinterpret_cast<uint4 *>(sA + a_off(m, 16)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            *reinterpret_cast<uint4 *>(sA + a_off(m, 24)) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
        };
        auto wait_acc = [&](int l, int i) {
            const bool ok = __all_sync(0xffffffffu, mbar_wait_cluster(&accfull[l], i & 1, wait_ns));
            tc_fence_after();
            return ok;
        };
        // a hidden layer: bias, tanh, FP16 into A chunk by chunk, each chunk signalled as round j at
        // once; the next chunk's TMEM load is in flight while one chunk is processed
        auto hidden = [&](uint32_t region, const float *bias) {
            const uint32_t tb = tmem + lane_addr + region * 256 + cq * 64;
            uint32_t cur[16];
            tmem_ld16_async(tb, cur);
            tmem_wait(cur);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t nxt[16];
                if (j < 3)
                    tmem_ld16_async(tb + 16 * (j + 1), nxt);
                const int col = cq * 64 + 16 * j;
                uint32_t p[8];
#pragma unroll
                for (int e = 0; e < 16; e += 2)
                    p[e >> 1] = pack2(tanh_fast(__uint_as_float(cur[e]) + bias[col + e]),
                                      tanh_fast(__uint_as_float(cur[e + 1]) + bias[col + e + 1]));
                *reinterpret_cast<uint4 *>(sA + a_off(m, col)) = make_uint4(p[0], p[1], p[2], p[3]);
                *reinterpret_cast<uint4 *>(sA + a_off(m, col + 8)) = make_uint4(p[4], p[5], p[6], p[7]);
                signal(j);
                if (j < 3) {
                    tmem_wait(nxt);
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        cur[e] = nxt[e];
                }
            }
        };
        bool ok = true;
        if (pair < ntiles) {
            if (cq == 0)
                write_x(pair);
            signal(0);  // every warp: round 0 counts all sixteen
        }
        int i = 0;
        for (int t = pair; t < ntiles; t += npairs, ++i) {
            if (*abort_flag || !wait_acc(0, i)) {
                ok = false;
                break;
            }
            hidden((3 * i) & 1, sb);
            if (*abort_flag || !wait_acc(1, i)) {
                ok = false;
                break;
            }
            hidden((3 * i + 1) & 1, sb + TCH);
            if (*abort_flag || !wait_acc(2, i)) {
                ok = false;
                break;
            }
            // A is free (layer 3's products are done): the next tile's inputs go in now
            if (t + npairs < ntiles) {
                if (cq == 0)
                    write_x(t + npairs);
                signal(0);
            }
            // layer 3: bias, tanh, and the 256 -> 2 output layer over this warp's 64 columns
            const uint32_t tb = tmem + lane_addr + ((3 * i + 2) & 1) * 256 + cq * 64;
            float y0 = 0.f, y1 = 0.f;
            uint32_t cur[16];
            tmem_ld16_async(tb, cur);
            tmem_wait(cur);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t nxt[16];
                if (j < 3)
                    tmem_ld16_async(tb + 16 * (j + 1), nxt);
                const int col = cq * 64 + 16 * j;
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const float h = tanh_fast(__uint_as_float(cur[e]) + sb[2 * TCH + col + e]);
                    y0 = fmaf(sW4[col + e], h, y0);
                    y1 = fmaf(sW4[TCH + col + e], h, y1);
                }
                if (j < 3) {
                    tmem_wait(nxt);
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        cur[e] = nxt[e];
                }
            }
            float2 *pp = part + (i & 1) * 4 * TROWS;
            pp[cq * TROWS + m] = make_float2(y0, y1);
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&bars[B_Y]);
            if (cq == 0) {
                if (!__all_sync(0xffffffffu, mbar_wait(&bars[B_Y], i & 1, wait_ns))) {
                    ok = false;
                    break;
                }
                const long row = (long)t * 2 * TROWS + rank * TROWS + m;
                if (row < n) {
                    const float2 a = pp[m], b = pp[TROWS + m], c = pp[2 * TROWS + m], e = pp[3 * TROWS + m];
                    Y[2 * row] = ((a.x + b.x) + c.x) + e.x + sb4[0];
                    Y[2 * row + 1] = ((a.y + b.y) + c.y) + e.y + sb4[1];
                }
            }
        }
        if (!ok && lane == 0) {
            record_error(err, GW_E_TIMEOUT, SITE_HERK_EPILOGUE, blockIdx.x);
            *abort_flag = 1;
        }
    }

    // ---------------- drain, then release TMEM and leave together
    __syncthreads();
    if (tid == 0) {
        if (!mbar_wait_cluster(&bars[B_DONE], 0, DRAIN_NS))
            record_error(err, GW_E_TIMEOUT, SITE_HERK_DRAIN, blockIdx.x);
        // the weight copies must land before the CTA leaves
        if (!*w_landed && !mbar_wait(&bars[B_W], 0, DRAIN_NS))
            record_error(err, GW_E_TIMEOUT, SITE_HERK_DRAIN, blockIdx.x);
    }
    tc_fence_before();
    cluster_sync_all();
    if (warp == CTRL_WARP) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, 512);
    }
    cluster_sync_all();
}

}  // namespace

size_t mlp_tc_weights_bytes()
{
    return WT_BYTES;
}

cudaError_t launch_mlp_tile_weights(const __half *W1, int n_in, const __half *W2, const __half *W3, uint8_t *Wt,
                                    cudaStream_t s)
{
    if (n_in < 1 || n_in > MAX_IN)
        return cudaErrorInvalidValue;
    tile_weights_kernel<<<128, 256, 0, s>>>(W1, n_in, W2, W3, Wt);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mlp_tc_forward(const float *X, long n, int n_in, const uint8_t *Wt, const float *b1,
                                  const float *b2, const float *b3, const __half *W4, const float *b4, float *Y,
                                  int num_sms, uint32_t *err, uint64_t wait_ns, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    if (n_in < 1 || n_in > MAX_IN || num_sms < 2)
        return cudaErrorInvalidValue;
    const long ntiles = (n + 2 * TROWS - 1) / (2 * TROWS);
    if (ntiles > (1L << 30))
        return cudaErrorInvalidValue;
    const int npairs = (int)std::min<long>(ntiles, num_sms / 2);
    cudaError_t e = cudaFuncSetAttribute(mlp_tc_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    if (e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * npairs, 1, 1);
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
    e = cudaLaunchKernelEx(&cfg, mlp_tc_pair_kernel, X, n, n_in, Wt, b1, b2, b3, W4, b4, Y, err, wait_ns);
    if (e != cudaSuccess)
        return e;
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gw
