// Tensor-core products of the correction network's training step: the hidden layers' forward
// products, the deltas back through W2 and W3, and the weight gradients of W1, W2 and W3.
//
// Precision: every FP32 operand is split into three BF16 parts, x = hi + mid + lo (exact: each
// part takes the next 8 bits of the significand, and BF16 has the FP32 exponent range), and a
// product takes the six part pairs down to 2^-16 (hi hi, hi mid, mid hi, hi lo, lo hi, mid mid):
// what is dropped is below 2^-24 of the product, so the result has FP32 accuracy with the FP32
// accumulation of tcgen05.mma kind::f16 (BF16 operands).
//
// Operand layout in global memory ("blocks"): an operand with R rows and K columns is cut into
// blocks of 128 rows x 16 k, block (kc, rb) at ((kc * nRB + rb) * 12 KB), each the three parts
// (4 KB each) in the K-major canonical layout of 8-row x 16-byte core matrices (128 bytes apart
// along K, 256 along the rows).  Rows beyond R and k beyond K are zero.  pack3_kernel writes a
// row-major FP32 matrix in this layout both ways: rows = its rows (the operand of a layer's
// product) and rows = its columns (the operand of a weight gradient, K = the batch).
//
// mlp_gemm3_kernel: C(m, n) = sum_k A(m, k) B(n, k) over one slice of K, one 128 x 128 tile per
// CTA; warp 0 streams the blocks with 1-D bulk copies into six 24 KB stages, warp 1 issues the six
// MMAs per 16-k chunk into TMEM, warps 2..9 read the tile and apply the epilogue: store a partial
// product (weight gradients, summed over slices afterwards), bias + tanh (forward) or times
// 1 - H^2 (back through tanh), and write the result also as the next products' operands (row and
// transposed, staged in the idle pipeline buffers) and its column sums.  Every wait is bounded.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "gw_internal.cuh"
#include "ptx.cuh"

namespace gw {

namespace {

constexpr int TR = 128;                    // rows of a block, and each side of a tile
constexpr int NPL = 3;                     // BF16 parts: hi, mid, lo
constexpr uint32_t PLB = TR * 16 * 2;      // 4 KB: one part of one block
constexpr uint32_t BLK = NPL * PLB;        // 12 KB: one block
constexpr int STAGES = 6;
constexpr uint32_t STAGE = 2 * BLK;        // 24 KB: a block of A and one of B
constexpr uint32_t PIPE = STAGES * STAGE;  // 144 KB
constexpr size_t SMEM = PIPE + 256;
constexpr int NEPI = 8;                    // epilogue warps: two per TMEM lane quarter
constexpr int NTHREADS = (2 + NEPI) * 32;  // warp 0 copies, warp 1 MMAs, warps 2..9 epilogue
constexpr uint64_t DRAIN_NS = 2000000000ull;
constexpr int PACK_PITCH = TR + 1;
constexpr int PACK_THREADS = 512;
constexpr size_t PACK_SMEM = (size_t)TR * PACK_PITCH * sizeof(float);
static_assert(PACK_SMEM <= PIPE, "the epilogue stages a tile in the pipeline buffers");

__host__ __device__ constexpr uint32_t blk_off(int r, int k)  // r < 128, k < 16
{
    return (r >> 3) * 256 + ((k >> 3) & 1) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ void named_bar_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void split3(float x, uint16_t &h, uint16_t &m, uint16_t &l)
{
    const __nv_bfloat16 bh = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(bh);
    const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(bm);
    h = __bfloat16_as_ushort(bh);
    m = __bfloat16_as_ushort(bm);
    l = __bfloat16_as_ushort(__float2bfloat16_rn(r2));
}

// 16 values of one row into the three parts of a block (k 0..15 of row r)
__device__ __forceinline__ void store_row16(uint8_t *blk, int r, const float *v)
{
    uint32_t w[NPL][8];
#pragma unroll
    for (int e = 0; e < 16; e += 2) {
        uint16_t h0, m0, l0, h1, m1, l1;
        split3(v[e], h0, m0, l0);
        split3(v[e + 1], h1, m1, l1);
        w[0][e >> 1] = h0 | ((uint32_t)h1 << 16);
        w[1][e >> 1] = m0 | ((uint32_t)m1 << 16);
        w[2][e >> 1] = l0 | ((uint32_t)l1 << 16);
    }
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
        *reinterpret_cast<uint4 *>(blk + p * PLB + blk_off(r, 0)) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
        *reinterpret_cast<uint4 *>(blk + p * PLB + blk_off(r, 8)) = make_uint4(w[p][4], w[p][5], w[p][6], w[p][7]);
    }
}

// One 128 x 128 tile (rows r0.., columns c0..) of the FP32 matrix S (row r at S + (rows ? rows[r] :
// r) * ld) into rowop (rows r, k = c; nRB = ceil(R / 128) row blocks, ceil(C / 16) chunks) and
// colop (rows c, k = r; ceil(C / 128) row blocks, ceil(R / 16) chunks).  Either may be null.
// colsum (if given): colsum[rb][c] = the sum of the tile's rows of column c (rb = r0 / 128).
// 512 threads; the loads cover only the tile's rows and columns in range (a narrow matrix such
// as the 12 input features takes 12 loads per row, not 128), the rest of the tile is zero.
__global__ void __launch_bounds__(PACK_THREADS) pack3_kernel(const float *__restrict__ S, long ld,
                                                             const int *__restrict__ rows, int R, int C,
                                                             uint8_t *__restrict__ rowop, uint8_t *__restrict__ colop,
                                                             float *__restrict__ colsum)
{
    extern __shared__ float tile[];  // [128][PACK_PITCH]
    const int r0 = blockIdx.y * TR, c0 = blockIdx.x * TR, t = threadIdx.x;
    const int rw = min(TR, R - r0), cw = min(TR, C - c0);  // rows and columns in range
    for (int e = t; e < TR * TR; e += PACK_THREADS)
        tile[(e >> 7) * PACK_PITCH + (e & 127)] = 0.f;
    __syncthreads();
    const int nv = rw * cw;
#pragma unroll 4
    for (int e = t; e < nv; e += PACK_THREADS) {
        const int i = e / cw, c = e - i * cw, r = r0 + i;
        tile[i * PACK_PITCH + c] = S[(long)(rows ? rows[r] : r) * ld + c0 + c];
    }
    __syncthreads();
    if (colsum && t < cw) {
        float acc = 0.f;
#pragma unroll 8
        for (int i = 0; i < TR; ++i)
            acc += tile[i * PACK_PITCH + t];
        colsum[(long)(r0 >> 7) * C + c0 + t] = acc;
    }
    if (rowop) {
        const int nrb = (R + TR - 1) / TR, nkc = (C + 15) / 16;
        for (int it = t; it < 8 * TR; it += PACK_THREADS) {
            const int row = it & 127, j = it >> 7;
            if ((c0 >> 4) + j >= nkc)
                continue;
            float v[16];
#pragma unroll
            for (int e = 0; e < 16; ++e)
                v[e] = tile[row * PACK_PITCH + j * 16 + e];
            store_row16(rowop + ((size_t)((c0 >> 4) + j) * nrb + (r0 >> 7)) * BLK, row, v);
        }
    }
    if (colop) {
        const int nrb = (C + TR - 1) / TR, nkc = (R + 15) / 16;
        for (int it = t; it < 8 * TR; it += PACK_THREADS) {
            const int col = it & 127, j = it >> 7;
            if ((r0 >> 4) + j >= nkc)
                continue;
            float v[16];
#pragma unroll
            for (int e = 0; e < 16; ++e)
                v[e] = tile[(j * 16 + e) * PACK_PITCH + col];
            store_row16(colop + ((size_t)((r0 >> 4) + j) * nrb + (c0 >> 7)) * BLK, col, v);
        }
    }
}

// The three weight matrices W_l (out x in, flat at w + off[l]) written element by element into their
// row operands (rows = outputs, k = inputs) and, for l = 1, 2, their transposes (rows = inputs).
// Padding (k beyond in, rows beyond out) is never written: the buffers are cleared once.
__global__ void pack_weights_kernel(const float *__restrict__ w, MlpWeightPack p)
{
    const long n0 = (long)p.hidden * p.n_in, n1 = (long)p.hidden * p.hidden, total = n0 + 2 * n1;
    const int nrb = (p.hidden + TR - 1) / TR;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int l = i < n0 ? 0 : (i < n0 + n1 ? 1 : 2);
        const long e = l == 0 ? i : i - n0 - (l - 1) * n1;
        const int in = l == 0 ? p.n_in : p.hidden;
        const int o = (int)(e / in), c = (int)(e - (long)o * in);
        uint16_t h, m, lo;
        split3(w[p.off[l] + e], h, m, lo);
        uint8_t *b = p.row[l] + ((size_t)(c >> 4) * nrb + (o >> 7)) * BLK + blk_off(o & 127, c & 15);
        *reinterpret_cast<uint16_t *>(b) = h;
        *reinterpret_cast<uint16_t *>(b + PLB) = m;
        *reinterpret_cast<uint16_t *>(b + 2 * PLB) = lo;
        if (l > 0) {
            uint8_t *bt = p.col[l - 1] + ((size_t)(o >> 4) * nrb + (c >> 7)) * BLK + blk_off(c & 127, o & 15);
            *reinterpret_cast<uint16_t *>(bt) = h;
            *reinterpret_cast<uint16_t *>(bt + PLB) = m;
            *reinterpret_cast<uint16_t *>(bt + 2 * PLB) = lo;
        }
    }
}

template <int EPI>
__global__ void __launch_bounds__(NTHREADS, 1)
    mlp_gemm3_kernel(const uint8_t *__restrict__ A, int nmb, const uint8_t *__restrict__ B, int nnb, int nkc, int kcs,
                     int M, int N, float *__restrict__ C, long ldc, long zstride, const float *__restrict__ bias,
                     const float *__restrict__ H, long ldh, uint8_t *__restrict__ rowop, uint8_t *__restrict__ colop,
                     float *__restrict__ colsum, uint32_t *err, uint64_t wait_ns)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + PIPE);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(accf + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    volatile int *n_issued = abort_flag + 1;
    volatile int *n_consumed = abort_flag + 2;
    volatile int *epi_ok = abort_flag + 3;  // [NEPI] each epilogue warp's wait result

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = blockIdx.x, mb = blockIdx.y, z = blockIdx.z;
    const int k0 = z * kcs, nch = max(0, min(nkc, k0 + kcs) - k0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accf, 1);
        *abort_flag = 0;
        *n_issued = 0;
        *n_consumed = 0;
        fence_barrier_init();
    }
    if (warp == 1)
        tmem_alloc(tslot, TR);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            for (int i = 0; i < nch; ++i) {
                const int s = i % STAGES;
                if (i >= STAGES && !mbar_wait(&empty[s], ((i / STAGES) - 1) & 1, wait_ns)) {
                    record_error(err, GW_E_TIMEOUT, SITE_HERK_PRODUCER, blockIdx.x);
                    *abort_flag = 1;
                    break;
                }
                if (*abort_flag)
                    break;
                uint8_t *st = smem + s * STAGE;
                mbar_arrive_expect_tx(&full[s], STAGE);
                bulk_g2s(st, A + ((size_t)(k0 + i) * nmb + mb) * BLK, BLK, &full[s]);
                bulk_g2s(st + BLK, B + ((size_t)(k0 + i) * nnb + nb) * BLK, BLK, &full[s]);
                *n_issued = i + 1;
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t ID = mma_idesc(1, TR, TR, false);  // BF16 x BF16, M 128, N 128
            constexpr uint64_t DP = PLB >> 4, DB = BLK >> 4, DS = STAGE >> 4;
            const uint64_t d0 = smem_desc(smem_u32(smem), 128, 256);
            for (int i = 0; i < nch; ++i) {
                const int s = i % STAGES;
                if (!mbar_wait(&full[s], (i / STAGES) & 1, wait_ns)) {
                    record_error(err, GW_E_TIMEOUT, SITE_HERK_MMA, blockIdx.x);
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint64_t a = d0 + (uint64_t)s * DS, b = a + DB;
                mma_f16(tmem, a, b, ID, i > 0 ? 1u : 0u);  // hi hi
                mma_f16(tmem, a, b + DP, ID, 1);            // hi mid
                mma_f16(tmem, a + DP, b, ID, 1);            // mid hi
                mma_f16(tmem, a, b + 2 * DP, ID, 1);        // hi lo
                mma_f16(tmem, a + 2 * DP, b, ID, 1);        // lo hi
                mma_f16(tmem, a + DP, b + DP, ID, 1);       // mid mid
                mma_commit(&empty[s]);
                *n_consumed = i + 1;
            }
            mma_commit(accf);  // arrives once every MMA issued above has completed
        }
        __syncwarp();
    } else {
        // epilogue warps 2..9: TMEM lane quarter warp & 3 (one tile row per lane), column half hf
        const int ew = warp - 2, q = warp & 3, hf = ew >> 2, rl = q * 32 + lane, m = mb * TR + rl;
        const int et = ew * 32 + lane;  // 0 .. 255
        const bool wok = __all_sync(0xffffffffu, mbar_wait(accf, 0, wait_ns));
        if (lane == 0) {
            epi_ok[ew] = (wok && *abort_flag == 0) ? 1 : 0;
            if (!wok)
                record_error(err, GW_E_TIMEOUT, SITE_HERK_EPILOGUE, blockIdx.x);
        }
        // every epilogue warp's wait has ended (each is bounded): one decision, from the same votes,
        // for all eight warps, so that all or none of them reach the staging barrier below
        named_bar_sync(1, NEPI * 32);
        bool ok = true;
#pragma unroll
        for (int w = 0; w < NEPI; ++w)
            ok = ok && epi_ok[w] != 0;
        if (!ok) {
            if (lane == 0)
                *abort_flag = 1;
        } else {
            tc_fence_after();
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16);
            float *crow = C + (EPI == 0 ? (long)z * zstride : 0) + (long)m * ldc;
            // 16-byte alignment of every row start of C (and H), and of bias
            const bool vec = ((reinterpret_cast<uintptr_t>(C) | (uintptr_t)(ldc * 4) | (uintptr_t)(zstride * 4) |
                               reinterpret_cast<uintptr_t>(bias) | reinterpret_cast<uintptr_t>(H) | (uintptr_t)(ldh * 4)) &
                              15) == 0;
            // the pipeline is idle (every MMA has completed): it stages the tile for colop / colsum
            float *stile = reinterpret_cast<float *>(smem);
            const bool stage = colop || colsum;
            const int nrb_m = (M + TR - 1) / TR, nrb_n = (N + TR - 1) / TR;
            const int nkc_n = (N + 15) / 16, nkc_m = (M + 15) / 16;
            for (int c0 = hf * 64; c0 < hf * 64 + 64; c0 += 16) {
                float v[16];
                if (nch > 0) {
                    tmem_ld16(taddr + c0, v);
                } else {
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        v[e] = 0.f;
                }
                const int n0 = nb * TR + c0;
                if (m < M && vec && n0 + 16 <= N) {
                    // whole 16-column group in range, rows 16-byte aligned: vector loads / stores
#pragma unroll
                    for (int e = 0; e < 16; e += 4) {
                        float4 x = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
                        if (EPI == 1) {
                            const float4 b = *reinterpret_cast<const float4 *>(bias + n0 + e);
                            x = make_float4(tanhf(x.x + b.x), tanhf(x.y + b.y), tanhf(x.z + b.z), tanhf(x.w + b.w));
                        } else if (EPI == 2) {
                            const float4 h = *reinterpret_cast<const float4 *>(H + (long)m * ldh + n0 + e);
                            x = make_float4(x.x * (1.f - h.x * h.x), x.y * (1.f - h.y * h.y),
                                            x.z * (1.f - h.z * h.z), x.w * (1.f - h.w * h.w));
                        }
                        *reinterpret_cast<float4 *>(crow + n0 + e) = x;
                        v[e] = x.x;
                        v[e + 1] = x.y;
                        v[e + 2] = x.z;
                        v[e + 3] = x.w;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int n = n0 + e;
                        float x = 0.f;  // rows and columns out of range stay zero in the packs
                        if (m < M && n < N) {
                            x = v[e];
                            if (EPI == 1)
                                x = tanhf(x + bias[n]);
                            else if (EPI == 2) {
                                const float h = H[(long)m * ldh + n];
                                x *= 1.f - h * h;
                            }
                            crow[n] = x;
                        }
                        v[e] = x;
                    }
                }
                // this row's 16 values as k chunk n0 / 16 of the row operand (rows m, k = n)
                if (rowop && (n0 >> 4) < nkc_n)
                    store_row16(rowop + ((size_t)(n0 >> 4) * nrb_m + mb) * BLK, rl, v);
                if (stage) {
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        stile[rl * PACK_PITCH + c0 + e] = v[e];
                }
            }
            if (stage) {
                named_bar_sync(1, NEPI * 32);
                // thread et now takes column cl of the tile, chunks 4 jh .. 4 jh + 3 of the transpose
                const int cl = et & 127, jh = et >> 7, n = nb * TR + cl;
                if (colop)
                    for (int j = 4 * jh; j < 4 * jh + 4 && mb * 8 + j < nkc_m; ++j) {
                        float v[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            v[e] = stile[(j * 16 + e) * PACK_PITCH + cl];
                        store_row16(colop + ((size_t)(mb * 8 + j) * nrb_n + nb) * BLK, cl, v);
                    }
                if (colsum && jh == 0 && n < N) {
                    float acc = 0.f;
#pragma unroll 8
                    for (int i = 0; i < TR; ++i)
                        acc += stile[i * PACK_PITCH + cl];
                    colsum[(long)mb * N + n] = acc;
                }
            }
        }
    }

    // ---------------- drain: every MMA done, every issued copy landed, then release TMEM
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!mbar_wait(accf, 0, DRAIN_NS))
            record_error(err, GW_E_TIMEOUT, SITE_HERK_DRAIN, blockIdx.x);
        const int issued = *n_issued, consumed = *n_consumed;
        for (int i = consumed; i < issued; ++i)
            if (!mbar_wait(&full[i % STAGES], (i / STAGES) & 1, DRAIN_NS)) {
                record_error(err, GW_E_TIMEOUT, SITE_HERK_DRAIN, blockIdx.x);
                break;
            }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, TR);
    }
}

}  // namespace

size_t mlp_pack3_bytes(int rows, int k)
{
    return (size_t)((rows + TR - 1) / TR) * ((k + 15) / 16) * BLK;
}

cudaError_t launch_mlp_pack3(const float *S, long ld, const int *rows, int R, int C, uint8_t *rowop, uint8_t *colop,
                             float *colsum, cudaStream_t s)
{
    if (R <= 0 || C <= 0)
        return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(pack3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PACK_SMEM);
    if (e != cudaSuccess)
        return e;
    const dim3 grid((C + TR - 1) / TR, (R + TR - 1) / TR);
    pack3_kernel<<<grid, PACK_THREADS, PACK_SMEM, s>>>(S, ld, rows, R, C, rowop, colop, colsum);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mlp_pack_weights(const float *w, const MlpWeightPack &p, int num_sms, cudaStream_t s)
{
    const long total = (long)p.hidden * p.n_in + 2L * p.hidden * p.hidden;
    const int blocks = (int)std::max(1L, std::min((total + 255) / 256, 4L * num_sms));
    pack_weights_kernel<<<blocks, 256, 0, s>>>(w, p);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mlp_gemm3(int epi, const uint8_t *A, int M, const uint8_t *B, int N, int K, int splits, float *C,
                             long ldc, long zstride, const float *bias, const float *H, long ldh, uint8_t *rowop,
                             uint8_t *colop, float *colsum, uint32_t *err, uint64_t wait_ns, cudaStream_t s,
                             int *slices_used)
{
    if (M <= 0 || N <= 0 || K <= 0 || epi < 0 || epi > 2)
        return cudaErrorInvalidValue;
    if (epi == 0 && (rowop || colop || colsum))  // partial products are not packed
        return cudaErrorInvalidValue;
    const int nmb = (M + TR - 1) / TR, nnb = (N + TR - 1) / TR, nkc = (K + 15) / 16;
    const int S0 = std::max(1, std::min(splits, nkc));
    const int kcs = (nkc + S0 - 1) / S0, S = (nkc + kcs - 1) / kcs;
    if (slices_used)
        *slices_used = S;
    const dim3 grid(nnb, nmb, S);
    cudaError_t e = cudaSuccess;
    switch (epi) {
    case 0:
        e = cudaFuncSetAttribute(mlp_gemm3_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (e == cudaSuccess)
            mlp_gemm3_kernel<0><<<grid, NTHREADS, SMEM, s>>>(A, nmb, B, nnb, nkc, kcs, M, N, C, ldc, zstride, bias, H,
                                                             ldh, rowop, colop, colsum, err, wait_ns);
        break;
    case 1:
        e = cudaFuncSetAttribute(mlp_gemm3_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (e == cudaSuccess)
            mlp_gemm3_kernel<1><<<grid, NTHREADS, SMEM, s>>>(A, nmb, B, nnb, nkc, kcs, M, N, C, ldc, zstride, bias, H,
                                                             ldh, rowop, colop, colsum, err, wait_ns);
        break;
    default:
        e = cudaFuncSetAttribute(mlp_gemm3_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (e == cudaSuccess)
            mlp_gemm3_kernel<2><<<grid, NTHREADS, SMEM, s>>>(A, nmb, B, nnb, nkc, kcs, M, N, C, ldc, zstride, bias, H,
                                                             ldh, rowop, colop, colsum, err, wait_ns);
        break;
    }
    if (e != cudaSuccess)
        return e;
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gw
