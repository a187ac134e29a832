// Tensor-core inference of the correction network (n_in -> 256 -> 256 -> 256 -> 2, tanh).
//
// Two persistent kernels, each keeping one 256 x 256 FP16 weight matrix resident in shared memory
// (128 KB) and walking 128-row tiles of the input:
//   l12: layer 1 on CUDA cores (n_in <= 16 inputs), its tanh output rounded to FP16 into the
//        tcgen05 operand layout in shared memory; h1 W2^T as 16 MMAs (kind::f16, M 128, N 256,
//        K 16) into TMEM; bias + tanh, rounded to FP16 and stored to global memory already in
//        the operand layout, one 64 KB block per tile;
//   l34: one bulk copy per tile brings that block back; h2 W3^T into TMEM; bias + tanh in FP32,
//        and the 256 -> 2 output layer folded into the same pass over the accumulator.
// Operand layout (K-major, no swizzle): 16-wide K chunks, each made of 8-row x 16-byte core
// matrices, 128 bytes apart along K and 256 bytes apart along M / N.
#include <cuda_fp16.h>

#include "gw_internal.cuh"
#include "ptx.cuh"

namespace gw {

namespace {

constexpr int TCH = 256;                         // hidden width of the tensor-core path
constexpr int TROWS = 128;                       // rows per tile
constexpr int MAX_IN = 16;                       // inputs of layer 1 on this path
constexpr uint32_t A_CHUNK = TROWS * 16 * 2;     // 4 KB: 128 rows x 16 k, FP16
constexpr uint32_t W_CHUNK = TCH * 16 * 2;       // 8 KB: 256 rows x 16 k
constexpr uint32_t A_TILE = 16 * A_CHUNK;        // 64 KB
constexpr uint32_t W_TILE = 16 * W_CHUNK;        // 128 KB
constexpr uint32_t IDESC = mma_idesc(0, TROWS, TCH, false);
constexpr uint64_t DRAIN_NS = 2000000000ull;

__device__ __forceinline__ uint32_t a_off(int m, int k)
{
    return (k >> 4) * A_CHUNK + (m >> 3) * 256 + ((k >> 3) & 1) * 128 + (m & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t w_off(int n, int k)
{
    return (k >> 4) * W_CHUNK + (n >> 3) * 256 + ((k >> 3) & 1) * 128 + (n & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    const __half ha = __float2half_rn(a), hb = __float2half_rn(b);
    return (uint32_t)__half_as_ushort(ha) | ((uint32_t)__half_as_ushort(hb) << 16);
}

// Row-major FP16 weights W [256][256] (out x in) -> operand layout (N = out, K = in).
__global__ void tile_weights_kernel(const __half *__restrict__ W, uint8_t *__restrict__ Wt)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < TCH * TCH; t += gridDim.x * blockDim.x) {
        const int n = t / TCH, k = t - n * TCH;
        *reinterpret_cast<__half *>(Wt + w_off(n, k)) = W[t];
    }
}

// 16 MMAs over K = 256 from one thread, then a commit to `bar`.
__device__ __forceinline__ void issue_tile_mma(uint32_t tmem, uint32_t sa, uint32_t sw, uint64_t *bar)
{
#pragma unroll
    for (int c = 0; c < 16; ++c)
        mma_f16(tmem, smem_desc(sa + c * A_CHUNK, 128, 256), smem_desc(sw + c * W_CHUNK, 128, 256), IDESC,
                c > 0 ? 1u : 0u);
    mma_commit(bar);
}

__global__ void __launch_bounds__(256, 1)
    mlp_tc_l12_kernel(const float *__restrict__ X, int n, int n_in, const __half *__restrict__ W1,
                      const float *__restrict__ b1, const uint8_t *__restrict__ W2t, const float *__restrict__ b2,
                      uint8_t *__restrict__ H2, uint32_t *err, uint64_t wait_ns)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sW = smem, *sA = smem + W_TILE;
    float *sW1 = reinterpret_cast<float *>(sA + A_TILE);  // [n_in][256]
    float *sb1 = sW1 + MAX_IN * TCH, *sb2 = sb1 + TCH;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sb2 + TCH);  // [0] weights, [1] products done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
    }
    if (warp == 0)
        tmem_alloc(tslot, 256);
    for (int t = tid; t < n_in * TCH; t += blockDim.x) {
        const int i = t / TCH, j = t - i * TCH;
        sW1[i * TCH + j] = __half2float(W1[j * n_in + i]);
    }
    for (int t = tid; t < TCH; t += blockDim.x) {
        sb1[t] = b1[t];
        sb2[t] = b2[t];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t sa = smem_u32(sA), sw = smem_u32(sW);
    if (tid == 0) {
        mbar_arrive_expect_tx(&bars[0], W_TILE);
        bulk_g2s(sW, W2t, W_TILE, &bars[0]);
    }
    bool ok = mbar_wait(&bars[0], 0, wait_ns);
    if (__syncthreads_or(!ok)) {
        if (tid == 0)
            record_error(err, GW_E_TIMEOUT, SITE_HERK_PRODUCER, blockIdx.x);
        mbar_wait(&bars[0], 0, DRAIN_NS);  // the weight copy must land before the CTA leaves
        ok = false;
    }
    const int ntiles = (n + TROWS - 1) / TROWS;
    int iter = 0;
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++iter) {
        // layer 1 on CUDA cores: row m, 128 of the 256 outputs per thread
        const int m = tid & 127, jh = (tid >> 7) * 128, row = tile * TROWS + m;
        float x[MAX_IN];
#pragma unroll
        for (int i = 0; i < MAX_IN; ++i)
            x[i] = (i < n_in && row < n) ? X[(size_t)row * n_in + i] : 0.f;
        for (int j0 = jh; j0 < jh + 128; j0 += 8) {
            uint32_t w4[4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                float acc0 = sb1[j0 + e], acc1 = sb1[j0 + e + 1];
#pragma unroll
                for (int i = 0; i < MAX_IN; ++i)
                    if (i < n_in) {
                        acc0 = fmaf(sW1[i * TCH + j0 + e], x[i], acc0);
                        acc1 = fmaf(sW1[i * TCH + j0 + e + 1], x[i], acc1);
                    }
                w4[e >> 1] = pack2(tanhf(acc0), tanhf(acc1));
            }
            *reinterpret_cast<uint4 *>(sA + a_off(m, j0)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
        fence_proxy_async_smem();  // the tensor core reads what the threads just wrote
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0)
            issue_tile_mma(tmem, sa, sw, &bars[1]);
        __syncwarp();
        ok = mbar_wait(&bars[1], iter & 1, wait_ns);
        if (__syncthreads_or(!ok)) {
            if (tid == 0)
                record_error(err, GW_E_TIMEOUT, SITE_HERK_MMA, blockIdx.x);
            mbar_wait(&bars[1], iter & 1, DRAIN_NS);
            ok = false;
            break;
        }
        tc_fence_after();
        // epilogue: warp -> TMEM lane quarter (32 rows) and column half
        const int q = warp & 3, ch = warp >> 2, mrow = q * 32 + lane;
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + ch * 128;
        uint8_t *dst = H2 + (size_t)tile * A_TILE;
        for (int c0 = 0; c0 < 128; c0 += 16) {
            float v[16];
            tmem_ld16(taddr + c0, v);
            const int j = ch * 128 + c0;
            uint32_t p[8];
#pragma unroll
            for (int e = 0; e < 16; e += 2)
                p[e >> 1] = pack2(tanhf(v[e] + sb2[j + e]), tanhf(v[e + 1] + sb2[j + e + 1]));
            *reinterpret_cast<uint4 *>(dst + a_off(mrow, j)) = make_uint4(p[0], p[1], p[2], p[3]);
            *reinterpret_cast<uint4 *>(dst + a_off(mrow, j + 8)) = make_uint4(p[4], p[5], p[6], p[7]);
        }
        tc_fence_before();
        __syncthreads();  // TMEM and the operand tile are free for the next tile
        tc_fence_after();
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 256);
    }
}

__global__ void __launch_bounds__(256, 1)
    mlp_tc_l34_kernel(const uint8_t *__restrict__ H2, int n, const uint8_t *__restrict__ W3t,
                      const float *__restrict__ b3, const __half *__restrict__ W4, const float *__restrict__ b4,
                      float *__restrict__ Y, uint32_t *err, uint64_t wait_ns)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sW = smem, *sA = smem + W_TILE;
    float *sb3 = reinterpret_cast<float *>(sA + A_TILE);
    float *sW4 = sb3 + TCH;                               // [2][256]
    float2 *part = reinterpret_cast<float2 *>(sW4 + 2 * TCH);  // [2][128] partial outputs per column half
    float *sb4 = reinterpret_cast<float *>(part + 2 * TROWS);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sb4 + 4);  // [0] weights, [1] tile, [2] products done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 3);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (n + TROWS - 1) / TROWS;
    if (tid == 0) {
        for (int b = 0; b < 3; ++b)
            mbar_init(&bars[b], 1);
        fence_barrier_init();
    }
    if (warp == 0)
        tmem_alloc(tslot, 256);
    for (int t = tid; t < TCH; t += blockDim.x) {
        sb3[t] = b3[t];
        sW4[t] = __half2float(W4[t]);
        sW4[TCH + t] = __half2float(W4[TCH + t]);
    }
    if (tid < 2)
        sb4[tid] = b4[tid];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t sa = smem_u32(sA), sw = smem_u32(sW);
    int issued = 0, consumed = 0;  // tile copies (thread 0's view)
    if (tid == 0) {
        mbar_arrive_expect_tx(&bars[0], W_TILE);
        bulk_g2s(sW, W3t, W_TILE, &bars[0]);
        if ((int)blockIdx.x < ntiles) {
            mbar_arrive_expect_tx(&bars[1], A_TILE);
            bulk_g2s(sA, H2 + (size_t)blockIdx.x * A_TILE, A_TILE, &bars[1]);
            issued = 1;
        }
    }
    bool ok = mbar_wait(&bars[0], 0, wait_ns);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            record_error(err, GW_E_TIMEOUT, SITE_HERK_PRODUCER, blockIdx.x);
            mbar_wait(&bars[0], 0, DRAIN_NS);  // the weight copy must land before the CTA leaves
        }
        ok = false;
    }
    int iter = 0;
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++iter) {
        ok = mbar_wait(&bars[1], iter & 1, wait_ns);
        if (__syncthreads_or(!ok)) {
            if (tid == 0)
                record_error(err, GW_E_TIMEOUT, SITE_HERK_PRODUCER, blockIdx.x);
            ok = false;
            break;
        }
        if (tid == 0)
            consumed = iter + 1;
        tc_fence_after();
        if (tid == 0)
            issue_tile_mma(tmem, sa, sw, &bars[2]);
        __syncwarp();
        ok = mbar_wait(&bars[2], iter & 1, wait_ns);
        if (__syncthreads_or(!ok)) {
            if (tid == 0)
                record_error(err, GW_E_TIMEOUT, SITE_HERK_MMA, blockIdx.x);
            mbar_wait(&bars[2], iter & 1, DRAIN_NS);
            ok = false;
            break;
        }
        tc_fence_after();
        // the operand tile is free once the products are done: fetch the next one meanwhile
        if (tid == 0 && tile + (int)gridDim.x < ntiles) {
            mbar_arrive_expect_tx(&bars[1], A_TILE);
            bulk_g2s(sA, H2 + (size_t)(tile + gridDim.x) * A_TILE, A_TILE, &bars[1]);
            issued = iter + 2;
        }
        const int q = warp & 3, ch = warp >> 2, mrow = q * 32 + lane;
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + ch * 128;
        float y0 = 0.f, y1 = 0.f;
        for (int c0 = 0; c0 < 128; c0 += 16) {
            float v[16];
            tmem_ld16(taddr + c0, v);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int j = ch * 128 + c0 + e;
                const float h = tanhf(v[e] + sb3[j]);
                y0 = fmaf(sW4[j], h, y0);
                y1 = fmaf(sW4[TCH + j], h, y1);
            }
        }
        part[ch * TROWS + mrow] = make_float2(y0, y1);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid < TROWS) {
            const int row = tile * TROWS + tid;
            if (row < n) {
                const float2 a = part[tid], b = part[TROWS + tid];
                Y[2 * (size_t)row] = a.x + b.x + sb4[0];
                Y[2 * (size_t)row + 1] = a.y + b.y + sb4[1];
            }
        }
        __syncthreads();  // part is rewritten by the next tile
    }
    // a tile copy still in flight (an early stop) must land before the CTA leaves
    if (tid == 0 && issued > consumed)
        mbar_wait(&bars[1], consumed & 1, DRAIN_NS);
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 256);
    }
}

constexpr size_t L12_SMEM = W_TILE + A_TILE + sizeof(float) * (MAX_IN * TCH + 2 * TCH) + 64;
constexpr size_t L34_SMEM = W_TILE + A_TILE + sizeof(float) * (3 * TCH) + sizeof(float2) * 2 * TROWS + 16 + 64;

}  // namespace

size_t mlp_tc_h2_bytes(int rows)
{
    return (size_t)((rows + TROWS - 1) / TROWS) * A_TILE;
}

cudaError_t launch_mlp_tile_weights(const __half *W, uint8_t *Wt, cudaStream_t s)
{
    tile_weights_kernel<<<64, 256, 0, s>>>(W, Wt);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mlp_tc_forward(const float *X, int n, int n_in, const __half *W1, const float *b1,
                                  const uint8_t *W2t, const float *b2, const uint8_t *W3t, const float *b3,
                                  const __half *W4, const float *b4, uint8_t *H2, float *Y, int num_sms,
                                  uint32_t *err, uint64_t wait_ns, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    if (n_in < 1 || n_in > MAX_IN)
        return cudaErrorInvalidValue;
    const int ntiles = (n + TROWS - 1) / TROWS, grid = ntiles < num_sms ? ntiles : num_sms;
    cudaError_t e = cudaFuncSetAttribute(mlp_tc_l12_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L12_SMEM);
    if (e != cudaSuccess)
        return e;
    e = cudaFuncSetAttribute(mlp_tc_l34_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L34_SMEM);
    if (e != cudaSuccess)
        return e;
    mlp_tc_l12_kernel<<<grid, 256, L12_SMEM, s>>>(X, n, n_in, W1, b1, W2t, b2, H2, err, wait_ns);
    mlp_tc_l34_kernel<<<grid, 256, L34_SMEM, s>>>(H2, n, W3t, b3, W4, b4, Y, err, wait_ns);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace gw
