// Internal declarations shared by the translation units of libgw.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <array>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gw.h"

namespace gw {

// Device status word layout: low byte = gw_status code, bits 8..15 = site, bits 16..31 =
// detail (tile or pivot index, saturated).  First error wins (atomicCAS from 0).
enum ErrSite : uint32_t {
    SITE_HERK_PRODUCER = 1,
    SITE_HERK_MMA = 2,
    SITE_HERK_EPILOGUE = 3,
    SITE_HERK_DRAIN = 4,
    SITE_CHOL_PIVOT = 5,
    SITE_INPUT = 6,
    SITE_ZGEMM = 7,
    SITE_NS = 8,
};

__device__ __forceinline__ void record_error(uint32_t *err, uint32_t code, uint32_t site, uint32_t detail)
{
    const uint32_t word = (code & 0xFFu) | ((site & 0xFFu) << 8) | ((detail > 0xFFFFu ? 0xFFFFu : detail) << 16);
    atomicCAS(err, 0u, word);
}

// Sphere/transform plan for one grid and one gcut (built on the host by this library).
struct DftPlan {
    int n[3];
    int ng;        // sphere size
    int c3;        // distinct m3 values used by the sphere
    int sym3;      // M when those values are exactly -M..M (in that order), else -1
    int cd;        // distinct (m2, m3) pairs used by the sphere
    int *m3list;   // [c3]   m3 values (device)
    int *disk;     // [cd*2] (m2, index into m3list) (device)
    int *gmap;     // [ng*2] (m1, index into disk) (device)
    int np2;       // disk pairs {(m2, m3), (-m2, m3)} when the disk is symmetric in m2, else 0
    int k2;        // max m2 of the disk
    int4 *pair2;   // [np2] (index into m3list, m2 >= 0, disk index of m2, of -m2 or -1 at m2 = 0)
    int np1;       // sphere pairs {(m1, m2, m3), (-m1, m2, m3)} (every sphere has them), else 0
    int k1;        // max m1 of the sphere
    int4 *pair1;   // [np1] (disk index, m1 >= 0, sphere index of m1, of -m1 or -1 at m1 = 0)
    float2 *tw;    // [n1 + n2 + n3] exp(+2 pi i t / n_a), FP64-derived (device)
    float2 *twc;   // the same table conjugated: exp(-2 pi i t / n_a)
};

// Plan of the one-kernel sphere transform (k_dft_fused.cu): tables of the sphere's m1, (m1, m2)
// disk and m3 ranges, and per-axis twiddles, for grids whose planes and rows are 16-byte multiples
// and spheres with max |m| <= 8.
struct FusedPlan {
    int n[3] = {0, 0, 0};
    int M = 0, ng = 0, cd = 0;
    std::vector<int> tab;     // integer tables (see k_dft_fused.cu)
    std::vector<float2> tw;   // (cos, sin) of 2 pi m j / n_a, m <= M, per axis
    int *d_tab = nullptr;     // device copies (inside a buffer the caller owns)
    float2 *d_tw = nullptr;
    bool ok = false;
    bool build(const int n[3], const std::vector<std::array<int, 3>> &sphere);
    size_t device_bytes() const;
    cudaError_t upload(void *dev, cudaStream_t s);
};

// Plasmon-pole workspace pieces (k_pp.cu) for N_g = ng and block b <= 40.
struct PPWork {
    double2 *S, *Om, *X, *Y, *T, *G, *U, *parts, *partsY, *rho, *rho2, *tw;
    double *theta, *res, *omega2;
    int *gvec, *flag;
    size_t bytes;
    static PPWork carve(void *base, int ng, int b, int nr);  // base == nullptr: sizes only
};

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string last_error;
    double wait_limit_ms = 2000.0;
    bool timing = false;
    cudaEvent_t ev[9] = {};
    unsigned ev_mask = 0;
    float times[6] = {};
    double times_sum[6] = {};
    long long times_n[6] = {};

    // problem
    bool loaded = false;
    int n1 = 0, n2 = 0, n3 = 0, nr = 0, nv = 0, nc = 0, nb = 0;
    double cell_L = 1.0;
    double q[3] = {0.0, 0.0, 0.0};  // wave vector of eps^q, in units of 2 pi / cell_L
    int k = 0, kpad = 0, nr_pad = 0;

    // device buffers (owned)
    uint32_t *d_err = nullptr;      // device status word
    float2 *d_psiT = nullptr;       // [nr][nb] complex64 (transposed states)
    double *d_E = nullptr;          // [nb] Hartree
    float *d_sw = nullptr;          // [nv][nc] sqrt(2/(Ec-Ev))
    float *d_F = nullptr;           // operand planes
    size_t F_bytes = 0;
    int F_prec = -1;
    float2 *d_P = nullptr;          // [nr][nr]
    size_t P_bytes = 0;
    bool P_ready = false;
    int2 *d_tiles = nullptr;        // HERK tile list
    int n_tiles = 0, tiles_rb = 0;
    int2 *d_tiles_g = nullptr;      // tile list of the N_g x N_g update (g-space route)
    int n_tiles_g = 0, tiles_g_pad = -1;
    float2 *d_PG_parts = nullptr;   // split-k partials of the N_g x N_g update

    // G space
    int gcut = -1, ng = 0;
    std::vector<int> gvec;          // host [ng*3]
    DftPlan plan = {};
    int *d_plan_mem = nullptr;
    FusedPlan fplan;                // the one-kernel sphere transform (fplan.ok = usable)
    int transform_kind = GW_TRANSFORM_TWO_KERNEL;
    void *d_fplan = nullptr;
    size_t cap_fplan = 0;
    float2 *d_Q = nullptr;          // [nr][ng]  row transform
    float2 *d_QT = nullptr;         // [ng][nr]  conj-transposed
    float2 *d_PG = nullptr;         // [ng][ng]
    float2 *d_PGsum = nullptr;      // running sum over k-points (gw_set_kweight)
    int PGsum_ng = -1;              // N_g of that sum (-1: none)
    double kweight = 1.0;           // weight of the next P~ (Sec. 4.1's 1/N_k)
    bool kaccumulate = false;       // add the next P~ to the running sum
    float2 *d_dftw = nullptr;       // sphere-transform workspace [rows][n1][cd]
    double *d_sv = nullptr;         // [ng] sqrt(V(G))
    size_t G_cap = 0;               // ng capacity of the G-space buffers
    bool PG_ready = false;

    // eps
    double2 *d_eps = nullptr;       // [ng][ng]
    double2 *d_epsinv = nullptr;    // [ng][ng]
    double2 *d_work = nullptr;      // workspace for the inverse
    double *d_scal = nullptr;       // FP64 scalars of the Newton iteration
    void *d_tcw = nullptr;          // workspace of the tensor-core Newton iteration / gw_zgemm_tc
    bool eps_ready = false;
    int newton_iters = 0;
    double tc_report[4] = {-1, -1, -1, -1};  // last tensor-core Newton inverse (gw_newton_tc_report)
    // gw_eps_inv's tensor-core inverse as a captured CUDA graph, valid for the key below
    cudaGraph_t ns_graph = nullptr;
    cudaGraphExec_t ns_exec = nullptr;
    cudaStream_t ns_cap_stream = nullptr;  // private stream the graph is captured on (never runs work)
    unsigned long long ns_graph_kernels = 0;
    struct NsKey {
        int n = 0;
        const void *A = nullptr, *X = nullptr, *work = nullptr, *err = nullptr;
        uint64_t wait_ns = 0;
        cudaStream_t s = nullptr;
        bool operator==(const NsKey &o) const
        {
            return n == o.n && A == o.A && X == o.X && work == o.work && err == o.err && wait_ns == o.wait_ns &&
                   s == o.s;
        }
    } ns_key;
    void *d_ppw = nullptr;          // plasmon-pole workspace
    PPWork pp = {};                 // its pieces (valid while pp_ready)
    int pp_b = 0, pp_nmodes = 0;
    bool pp_ready = false;

    // staging for gw_load_states
    float2 *d_psi = nullptr;        // [nb][nr] complex64
    double2 *d_psi128 = nullptr;    // complex128 input staging
    float2 *d_coef = nullptr;       // plane-wave coefficients [nb][npw] (gw_load_states_g)
    int *d_gidx = nullptr;          // their grid indices
    float2 *d_gtw = nullptr;        // twiddles of the three axes
    float2 *d_psig = nullptr;       // transform workspace [nb][nr]

    // allocation capacities in bytes (buffers are reused while large enough)
    struct {
        size_t psi, psi128, psiT, E, sw, F, P, tiles, tiles_g, PG_parts, plan, Q, QT, PG, dftw, sv, eps, epsinv, work,
            scal, tcw, PGsum, coef, gidx, gtw, psig, ppw;
    } cap = {};
    int tiles_nr_pad = -1, tiles_kind = -1;
    float sw_max = 0.f;             // max sqrt(2/(E_c - E_v)) (host, from the energies)
    unsigned *d_small = nullptr;    // [0] |f| bound bits, [1] FP16 scale exponent
    int herk_W = 3, herk_L = 256;   // 6.5e-7 against FP64 at 24^3; see gw_set_herk_window
    int herk_kernel = GW_HERK_SINGLE; // r-space 16-bit update: one CTA per tile or CTA pairs
    std::vector<double> E_h;        // the loaded energies in Hartree (host copy)
    float *d_csw = nullptr;         // closure pair weights [nv][nb], then [nv][nv] for the occupied pairs
    float2 *d_Qc = nullptr;         // closure matrix elements when built from gw_build_PG's transforms
    size_t cap_Qc = 0;
    bool q_pairs = false;           // d_Q holds gw_build_PG's pair transforms of the loaded states,
    int q_pairs_gen = -1;           // for the plan of this generation
    double *d_cw = nullptr;         // closure weights W_v / (N_r - nb) [nv]
    int *d_cgvec = nullptr;         // sphere vectors [ng][3] for the closure
    void *d_cwork = nullptr;        // closure workspace
    // closure uploads without a stream sync: the weights go through pinned staging, reused once the
    // event of the previous upload has passed; the twiddles and the sphere vectors go up once per
    // grid / plan (the buffers they went into, and for which grid or plan)
    float *h_csw = nullptr;
    double *h_cw = nullptr;
    size_t cap_hcsw = 0, cap_hcw = 0;
    cudaEvent_t ev_cstage = nullptr;
    bool cstage_pending = false;
    const void *ctw_buf = nullptr;
    int ctw_dims[3] = {0, 0, 0};
    const void *cgvec_buf = nullptr;
    int cgvec_gen = -1;
    int plan_gen = 0;               // incremented by every plan build
    size_t cap_csw = 0, cap_cw = 0, cap_cgvec = 0, cap_cwork = 0;
    int last_herk_kernel = -1;      // the kernel of the last 16-bit r-space update
    double err_target = 0.0;        // > 0: the window comes from gw_set_error_target's rule
    int last_W = 3;                 // the window of the last 16-bit rank-k update
    uint32_t last_status = 0;       // the device status word read by the last synchronising call

    void release();
};

// Process-wide count of kernels this library has launched (reported by gw_get_stats).
void count_launches(int n);

// ---- launchers (each returns cudaGetLastError() of its launches) ----

// k_pair.cu
cudaError_t launch_transpose_states(const float2 *psi, int nb, int nr, float2 *psiT, cudaStream_t s);
cudaError_t launch_c128_to_c64(const double2 *in, size_t n, float2 *out, cudaStream_t s);
cudaError_t launch_check_finite(const float2 *x, size_t n, uint32_t *err, cudaStream_t s);
cudaError_t launch_weights(const double *E, int nv, int nc, float *sw, cudaStream_t s);
// prec: 0 = TF32X3 planes, 2 = TF32X1 planes, 3 = plain complex64 [kpad][nr_pad]
// Plain complex64 pair densities f [rows][nr_pad] (rows >= nv nc; extra rows and columns zero),
// written with r contiguous through a shared-memory transpose.
cudaError_t launch_pair_density_rows(const float2 *psiT, const float *sw, int nr, int nb, int nv, int nc, int rows,
                                     int nr_pad, float2 *F, cudaStream_t s);
cudaError_t launch_pair_density(const float2 *psiT, const float *sw, int nr, int nb, int nv, int nc,
                                int kpad, int nr_pad, int prec, float *F, cudaStream_t s);

// k_herk.cu
size_t herk_smem_bytes(int prec);
cudaError_t launch_herk_tc(const float *F, int prec, int kpad, int nr, int nr_pad, const int2 *tiles,
                           int n_tiles, float2 *P, uint32_t *err, uint64_t wait_ns, cudaStream_t s);
cudaError_t launch_herk_simt(const float2 *F, int kpad, int nr, int nr_pad, float2 *P, cudaStream_t s);
constexpr int HERK_BM = 128;
constexpr int HERK_BN = 256;
constexpr int HERK_KC = 8;
constexpr int HERK16_KC = 16;
// 16-bit operand planes.  For every 16-wide chunk of k and every 128-row block of r, the block's
// planes are stored next to each other (4 KB each, canonical K-major core-matrix layout), so that
// one bulk copy fetches all of a block's planes for a chunk:
//   element (r, k) of plane slot p sits at 16-bit offset
//   ((kc * nblk + r / 128) * npl + p) * 2048 + ((r % 128) / 8) * 128 + ((k % 16) / 8) * 64
//       + (r % 8) * 8 + k % 8,          kc = k / 16, nblk = nr_pad / 128.
// Four planes (one CTA per tile): Im hi, Re hi, Im lo, Re lo, so that [Im; Re] of each part is
// one 256-row MMA operand.  Six planes (CTA pairs): Im hi, Im lo, Re hi, Re lo, -Im hi, -Im lo, so
// that the even CTA's operand is slots 0..3 and the odd CTA's slots 2..5.
constexpr int HERK16_NPL = 4;
constexpr int HERK16_NPL_PAIR = 6;
enum { P4_IH = 0, P4_RH = 1, P4_IL = 2, P4_RL = 3 };
enum { P6_IH = 0, P6_IL = 1, P6_RH = 2, P6_RL = 3, P6_NIH = 4, P6_NIL = 5 };
__host__ __device__ __forceinline__ size_t plane16_block(int kc, int blk, int nblk, int npl, int slot)
{
    return (((size_t)kc * nblk + blk) * npl + slot) * 2048;
}
constexpr int HERK16_T = 128;

// k_herk16.cu, k_planes16.cu
size_t herk16_smem_bytes();
// npl: planes per k chunk written, HERK16_NPL or HERK16_NPL_PAIR
cudaError_t launch_pair_density16(const float2 *psiT, const float *sw, float sw_max, int nr, int nb, int nv, int nc,
                                  int kpad, int nr_pad, bool bf16, unsigned *bound_bits, int *scale_exp, uint16_t *F,
                                  cudaStream_t s, int npl = HERK16_NPL);
// splits > 1 (with a workspace P_parts of splits x nr^2 complex64): split-k over blockIdx.y, for
// updates with too few tiles to fill the GPU; the partials are summed in a fixed order into P.
// npl: planes per block and k chunk of F (HERK16_NPL); cps: k chunks per pipeline stage (1..3, 0 =
// chosen from W)
cudaError_t launch_herk16(const uint16_t *F, bool bf16, int kpad, int nr, int nr_pad, const int2 *tiles, int n_tiles,
                          float2 *P, const int *scale_exp, uint32_t *err, uint64_t wait_ns, int W, int L,
                          cudaStream_t s, int splits = 1, float2 *P_parts = nullptr, int npl = HERK16_NPL,
                          int cps = 0);
// k_herk16x2.cu: the same update on CTA pairs (2-SM MMAs, 256 x 128 complex tiles); F must hold
// HERK16_NPL_PAIR planes per chunk and nr_pad must be a multiple of 256.
size_t herk16x2_smem_bytes();
std::vector<int2> herk_pair_tiles(int nr_pad);
cudaError_t launch_herk16x2(const uint16_t *F, bool bf16, int kpad, int nr, int nr_pad, const int2 *pair_tiles,
                            int n_pairs, float2 *P, const int *scale_exp, uint32_t *err, uint64_t wait_ns, int W, int L,
                            cudaStream_t s);
// 16-bit hi/lo operand planes of a complex64 matrix M[k][j] (k < rows, j < cols, row stride ld)
// for launch_herk16 with nr = cols, nr_pad = cols_pad; the scale exponent comes from max |M|.
cudaError_t launch_planes16_from_c64(const float2 *M, int rows, int cols, long ld, int kpad, int cols_pad, bool bf16,
                                     unsigned *bound_bits, int *scale_exp, uint16_t *F, cudaStream_t s);

// k_herk16p.cu: persistent multi-instance rank-k update.  One job per instance; tiles are
// (job, 128-row block of r, 128-row block of r', 0) in the order CTAs take them (tile t goes to
// CTA t mod grid).
struct HerkJob {
    const uint16_t *F;
    float2 *P;
    const int *scale_exp;
    int nr, nr_pad, kpad, pad;
};
cudaError_t launch_herk16p(const HerkJob *jobs, const int4 *tiles, int n_tiles, int grid, bool bf16, uint32_t *err,
                           uint64_t wait_ns, int W, int L, cudaStream_t s);

// k_mlp_tc.cu: tensor-core inference of the correction network (hidden width 256, n_in <= 16)
// on CTA pairs; the weights go through launch_mlp_tile_weights into a buffer of
// mlp_tc_weights_bytes() first.
size_t mlp_tc_weights_bytes();
cudaError_t launch_mlp_tile_weights(const __half *W1, int n_in, const __half *W2, const __half *W3, uint8_t *Wt,
                                    cudaStream_t s);
cudaError_t launch_mlp_tc_forward(const float *X, long n, int n_in, const uint8_t *Wt, const float *b1,
                                  const float *b2, const float *b3, const __half *W4, const float *b4, float *Y,
                                  int num_sms, uint32_t *err, uint64_t wait_ns, cudaStream_t s);

// k_mlp_train.cu: tensor-core products of the correction network's training step.  Operands in the
// three-part BF16 block layout (mlp_pack3_bytes(rows, k) bytes); launch_mlp_pack3 writes an FP32
// matrix S [R][C] (rows gathered by `rows` if given) as rowop (rows R, k = C) and/or colop (rows
// C, k = R) and, if colsum is given, the column sums of each 128-row tile to colsum[ceil(R/128)][C].
// launch_mlp_gemm3: C(m, n) = sum_k A(m, k) B(n, k) (M x N, K), epi 0 = partial products of up to
// `splits` slices of K at C + z * zstride, 1 = tanh(acc + bias[n]), 2 = acc * (1 - H(m, n)^2);
// the slice count used goes to *slices_used.
// launch_mlp_gemm3 with epi 1 or 2 also writes its result (M x N) to rowop (rows M, k = N), colop
// (rows N, k = M) and its column sums per 128-row tile to colsum, where given.
// launch_mlp_pack_weights: W1 (hidden x n_in), W2, W3 (hidden x hidden) at w + off[l] into row[l]
// (rows = outputs) and W2, W3 into col[0], col[1] (rows = inputs), element by element (the
// padding of these buffers is never written: clear them once).
struct MlpWeightPack {
    uint8_t *row[3];
    uint8_t *col[2];
    long off[3];
    int hidden, n_in;
};
size_t mlp_pack3_bytes(int rows, int k);
cudaError_t launch_mlp_pack_weights(const float *w, const MlpWeightPack &p, int num_sms, cudaStream_t s);
cudaError_t launch_mlp_pack3(const float *S, long ld, const int *rows, int R, int C, uint8_t *rowop, uint8_t *colop,
                             float *colsum, cudaStream_t s);
cudaError_t launch_mlp_gemm3(int epi, const uint8_t *A, int M, const uint8_t *B, int N, int K, int splits, float *C,
                             long ldc, long zstride, const float *bias, const float *H, long ldh, uint8_t *rowop,
                             uint8_t *colop, float *colsum, uint32_t *err, uint64_t wait_ns, cudaStream_t s,
                             int *slices_used);

// k_dft_fused.cu: the whole sphere transform of a row in one kernel (planes streamed by bulk
// copies, stages j1 -> m1, j2 -> m2, j3 -> m3 in shared memory), for grids whose planes and rows
// are 16-byte multiples and spheres with max |m| <= 8.
// rows of X [rows][ldx] (sw == nullptr), or the pair densities conj(psi_v) psi_c sw[k] of the states
// X = psi [nb][ldx] (k = v nc + c, psi_c at state c0 + c), to Y [rows][ldy] on the sphere.
// cudaErrorNotSupported (nothing launched) where the plan or the alignment does not allow it.
cudaError_t launch_dft_fused(const float2 *X, long long ldx, int rows, float2 *Y, long long ldy, const FusedPlan &p,
                             bool negative_exponent, const float *sw, int nv, int nc, int c0, uint32_t *err,
                             uint64_t wait_ns, cudaStream_t s);

// k_dft.cu
size_t dft_smem_bytes(const DftPlan &p, int rows_per_cta);
bool dft_supported(const DftPlan &p);  // sphere small enough for the transform kernel
// Two-kernel form with a workspace of dft_work_bytes(p, rows) (stages 1 and 2 per plane, stage 3
// per row).  const_twiddles: stages 1 and 2 with compile-time twiddles where the plan allows
// (square planes of a compiled size up to 27, spheres at q = 0 with max |m3| <= 7), else twiddle
// tables in shared memory.
size_t dft_work_bytes(const DftPlan &p, int rows);
cudaError_t launch_dft_rows_ws(const float2 *X, long long ldx, int rows, float2 *Y, long long ldy, const DftPlan &p,
                               float2 *work, cudaStream_t s, bool negative_exponent = false,
                               bool const_twiddles = true);
// The same transform of the nv nc pair densities f_k = conj(psi_v) psi_c sw[k] (k = v nc + c),
// formed from the states psi [nb][nr] inside the kernel; row k of Y is f_k's transform.
// cudaErrorNotSupported (nothing launched) where the grid needs the row-block kernel.
// c0: state index of the first c of the pairs (-1: nv, the unoccupied states).
cudaError_t launch_dft_pairs_ws(const float2 *psi, long long nr, const float *sw, int nv, int nc, float2 *Y,
                                long long ldy, const DftPlan &p, float2 *work, cudaStream_t s,
                                bool negative_exponent, int c0 = -1, bool const_twiddles = true);
// negative_exponent: exp(-iG.r) instead of exp(+iG.r) (the conjugated twiddle table)
cudaError_t launch_dft_rows(const float2 *X, long long ldx, int rows, float2 *Y, long long ldy,
                            const DftPlan &p, cudaStream_t s, bool negative_exponent = false);
cudaError_t launch_conj_transpose(const float2 *in, int rows, int cols, float2 *out, cudaStream_t s);
cudaError_t launch_hermitize(float2 *A, int n, cudaStream_t s);  // A <- (A + A^H) / 2

// k_eps.cu
cudaError_t launch_eps_build(const float2 *PG, const double *sv, int ng, double2 *eps, cudaStream_t s);
// C = alpha * op(A) * op(B) + beta * C, complex128 row-major; op: 0 = N, 1 = conj-transpose.
// flags: ZG_B_LOWER  op(B)[k][j] = 0 for k < j (skip those k);  ZG_A_UPPER  op(A)[i][k] = 0 for
// k < i;  ZG_C_LOWER  compute and store only C[i][j] with j <= i;  ZG_C_MIRROR  with ZG_C_LOWER,
// also store C[j][i] = conj(C[i][j]) (beta must be 0);  ZG_A_LOWER  op(A)[i][k] = 0 for k > i.
enum { ZG_B_LOWER = 1, ZG_A_UPPER = 2, ZG_C_LOWER = 4, ZG_C_MIRROR = 8, ZG_A_LOWER = 16 };
cudaError_t launch_zgemm(int M, int N, int K, double2 alpha, const double2 *A, int lda, int opA,
                         const double2 *B, int ldb, int opB, double2 beta, double2 *C, int ldc, cudaStream_t s,
                         int flags = 0);
// The same for `batch` independent products; problem z uses A + z sA, B + z sB, C + z sC.
cudaError_t launch_zgemm_batched(int M, int N, int K, double2 alpha, const double2 *A, int lda, int opA, long sA,
                                 const double2 *B, int ldb, int opB, long sB, double2 beta, double2 *C, int ldc,
                                 long sC, int batch, cudaStream_t s, int flags = 0);
cudaError_t launch_chol_diag(double2 *A, int lda, int n, double2 *Linv, int ldl, int pivot0, uint32_t *err,
                             cudaStream_t s);
// Enqueue eps^-1 = (L L^H)^-1 in FP64 (Cholesky, recursive-doubling triangular inverse, Y^H Y).
// Workspace: A, Y, T of N^2 complex128 each, W of 32 N, Dinv of ceil(N/32) 32^2.
cudaError_t chol_inverse_enqueue(const double2 *eps, int N, double2 *epsinv, double2 *A, double2 *Y, double2 *T,
                                 double2 *W, double2 *Dinv, uint32_t *err, cudaStream_t s);
cudaError_t launch_copy_block(const double2 *src, int lds, double2 *dst, int ldd, int rows, int cols,
                              cudaStream_t s);
cudaError_t launch_set_identity(double2 *A, int lda, int n, double scale, cudaStream_t s);
cudaError_t launch_two_minus(double2 *T, int n, cudaStream_t s);  // T <- 2I - T
cudaError_t launch_scaled_adjoint(const double2 *A, int n, const double *d_den, double2 *X, cudaStream_t s);
cudaError_t launch_max_absdiff(const double2 *A, const double2 *B, size_t n, double *out, cudaStream_t s);
cudaError_t launch_row_abs_sum_max(const double2 *A, int n, double *out, cudaStream_t s);

// k_zgemm16.cu: complex GEMM from sliced FP64 operands on the 16-bit tensor cores, and the
// tensor-core Newton iteration for eps^-1.
struct ZPlan {
    int mode = 0;  // 0 = FP16X3 split, 1 = integer slices (FP64 accuracy)
    int M = 0, N = 0, K = 0, Mpad = 0, Npad = 0, nkc = 0, ntiles = 0, nslots = 0, npairs = 0;
    int ns = 0;   // slices of B (and the pairs t + u < ns); FP16X3: 2 (hi, lo)
    int nsA = 0;  // slices held in the A planes (>= ns; the refinement reuses eps's nine)
    std::vector<int2> host_pairs;
    std::vector<int> host_slots, host_wexp;
    int2 *d_pairs = nullptr;
    int *d_slots = nullptr, *d_wexp = nullptr;
    void build(int mode, int M, int N, int K, int nsm, int slices = 0, int slicesA = 0);
    size_t table_bytes() const;
    size_t planes_bytes(bool a_operand) const;
    size_t T_bytes() const;
    cudaError_t upload(void *tab, cudaStream_t s);
};
size_t zgemm_work_bytes(const ZPlan &p);
// k_pp.cu: the plasmon-pole model of Sec. 5.2 (workspace struct PPWork above).
cudaError_t pp_prepare(const PPWork &w, const double2 *epsinv, const double *sv, const float2 *psiT, int ng, int nr,
                       int nb, int nv, const int dims[3], const int *gvec_host, double cell_L, const double q[3],
                       cudaStream_t s);
cudaError_t pp_iterate(PPWork &w, int ng, int b, int nmodes, double tol, int max_iter, int *iters_out,
                       cudaStream_t s);
cudaError_t pp_eval(const PPWork &w, int ng, int b, int nuse, double omega, double2 *Sout, cudaStream_t s);
// The band-truncation closure estimate (gw_corr_closure): rhoG = FP64 transform, on the whole grid,
// of rho_W(r) = sum_{v < nv} w[v] |psi_v(r)|^2 (work: 2 N_r double2 + 3 * 64 twiddles), then
// out(g, h) = rhoG((m_g - m_h) mod n) - Ph(g, h) as complex64.  closure_set_twiddles fills the
// twiddles of the grid into the workspace (synchronously, once per grid); closure_enqueue is
// asynchronous.
size_t closure_work_bytes(int nr);
cudaError_t closure_set_twiddles(const int dims[3], int nr, void *work, cudaStream_t s);
// Rows k = v nc + c of Q (the pair transforms of gw_build_PG, weighted sqrt(2/(E_c - E_v)) = sw[k])
// rescaled to the closure's weight csw[v nb]: out[k][g] = Q[k][g] csw[v nb] / sw[k], for k < nv nc.
cudaError_t launch_closure_rescale(const float2 *Q, int nv, int nc, int ng, const float *csw, int nb, const float *sw,
                                   float2 *out, cudaStream_t s);
cudaError_t closure_enqueue(const float2 *psiT, int nr, int nb, int nv, const double *w, const int dims[3],
                            const int *gvec_dev, int ng, const float2 *Ph, float2 *out, void *work,
                            cudaStream_t s);
// k_states.cu
cudaError_t launch_states_from_g(const float2 *coef, int nb, int npw, const int *idx, int n1, int n2, int n3,
                                 const float2 *tw, float2 *work, float2 *out, cudaStream_t s);
cudaError_t launch_kweight(float2 *PG, const float2 *sum, size_t n, float w, bool acc, cudaStream_t s);
cudaError_t zgemm_enqueue(ZPlan &p, const double2 *A, long lda, const double2 *B, long ldb, double2 *C, void *work,
                          uint32_t *err, uint64_t wait_ns, cudaStream_t s);
size_t ns_work_bytes(int N, int nsm);
cudaError_t ns_report(const void *work, int N, int nsm, double *out4);
cudaError_t ns_prepare(void *work, int N, int nsm, cudaStream_t s);
// max_steps: FP16X3 Newton steps queued in the graph-safe form (at most 16, the eager form's limit).
// A last residual above the acceptance bar is GW_E_NUMERIC at SITE_NS with detail NS_DETAIL_CAP
// when phase 1 had not converged within its steps (the eager form, with more steps, may), else 0.
constexpr int NS_GRAPH_STEPS = 8;   // the typical eps needs 5-6 from the Jacobi-scaled start
constexpr uint32_t NS_DETAIL_CAP = 1;
cudaError_t ns_inverse_enqueue(const double2 *A, int N, double2 *Xout, void *work, double *rowsum, uint32_t *err,
                               uint64_t wait_ns, int nsm, cudaStream_t s, bool graph_safe = false,
                               int max_steps = 16);

}  // namespace gw
