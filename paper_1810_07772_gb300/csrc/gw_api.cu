// C ABI of libgw: context management, argument checks and the host-side orchestration of the
// kernels of the static-polarizability path (Kim et al., arXiv 1810.07772, Sec. 4.1 and 5.1).
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "gw_internal.cuh"

using namespace gw;

namespace gw {
void count_launches(int n);
}

struct gw_ctx {
    Ctx c;
};

namespace {

constexpr double HARTREE_EV = 27.211386245988;
constexpr double PI = 3.14159265358979323846;
constexpr int CHOL_NB = 32;

template <typename T>
void dfree(T *&p)
{
    if (p)
        cudaFree(p);
    p = nullptr;
}

gw_status fail(Ctx &c, gw_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c.last_error = buf;
    return st;
}

gw_status cuda_fail(Ctx &c, cudaError_t e, const char *where)
{
    cudaGetLastError();  // clear a sticky-free error so the context stays usable
    if (e == cudaErrorMemoryAllocation)
        return fail(c, GW_E_NOMEM, "%s: out of device memory", where);
    return fail(c, GW_E_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define GW_CUDA(call, where)                \
    do {                                    \
        cudaError_t e_ = (call);            \
        if (e_ != cudaSuccess)              \
            return cuda_fail(c, e_, where); \
    } while (0)

#define GW_TRY(expr)                \
    do {                            \
        gw_status s_ = (expr);      \
        if (s_ != GW_OK)            \
            return s_;              \
    } while (0)

// (Re)allocate a device buffer if its capacity is below `bytes`; contents are not kept.
template <typename T>
gw_status ensure(Ctx &c, T *&p, size_t &cap, size_t bytes, const char *what)
{
    if (p && cap >= bytes)
        return GW_OK;
    dfree(p);
    cap = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&p), bytes ? bytes : 16);
    if (e != cudaSuccess) {
        p = nullptr;
        return cuda_fail(c, e, what);
    }
    cap = bytes;
    return GW_OK;
}

std::atomic<unsigned long long> g_launches{0};

// Kernel-boundary events: build_P 0..2, P_to_G 3..5, eps_inv 6..8.  Recording never blocks; the
// elapsed times are read at the next synchronisation (gw_eps_inv, gw_get_times).
void record(Ctx &c, int i)
{
    if (c.timing) {
        cudaEventRecord(c.ev[i], c.stream);
        c.ev_mask |= 1u << i;
    }
}

void resolve_times(Ctx &c)
{
    static const int pairs[6][2] = {{0, 1}, {1, 2}, {3, 4}, {4, 5}, {6, 7}, {7, 8}};
    unsigned used = 0;
    for (int t = 0; t < 6; ++t) {
        const unsigned need = (1u << pairs[t][0]) | (1u << pairs[t][1]);
        if ((c.ev_mask & need) == need) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, c.ev[pairs[t][0]], c.ev[pairs[t][1]]) == cudaSuccess) {
                c.times[t] = ms;
                c.times_sum[t] += ms;
                c.times_n[t] += 1;
            }
            used |= need;
        }
    }
    c.ev_mask &= ~used;  // events shared by two pairs are cleared only after both were read
    cudaGetLastError();
}

// Device status word -> gw_status (the word is cleared).
gw_status read_device_status(Ctx &c)
{
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "stream synchronize");
    uint32_t word = 0;
    e = cudaMemcpy(&word, c.d_err, sizeof word, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "status readback");
    c.last_status = word;
    if (word == 0)
        return GW_OK;
    cudaMemset(c.d_err, 0, sizeof(uint32_t));
    const uint32_t code = word & 0xFF, site = (word >> 8) & 0xFF, detail = word >> 16;
    static const char *sites[] = {"?",
                                  "rank-k update producer",
                                  "rank-k update MMA issuer",
                                  "rank-k update epilogue",
                                  "rank-k update drain",
                                  "Cholesky pivot",
                                  "input check",
                                  "sliced complex GEMM",
                                  "tensor-core Newton iteration"};
    const char *sname = site < sizeof(sites) / sizeof(sites[0]) ? sites[site] : "?";
    if (code == GW_E_NUMERIC && site == SITE_NS)
        return fail(c, GW_E_NUMERIC, "tensor-core Newton iteration: residual above 1e-8 before the last "
                                     "refinement (matrix not positive definite or too ill-conditioned%s)",
                    detail == NS_DETAIL_CAP ? "; the FP16X3 steps had not converged" : "");
    if (code == GW_E_NUMERIC)
        return fail(c, GW_E_NUMERIC, "eps is not positive definite: Cholesky pivot %u <= 0", detail);
    if (code == GW_E_INVALID)
        return fail(c, GW_E_INVALID, "non-finite value in the states (%s)", sname);
    return fail(c, static_cast<gw_status>(code), "device wait ran out in the %s (block %u)", sname, detail);
}

// Measured error of the FP16 split against FP64 on the 24^3 workload (k = 15360) for window
// lengths W (chunks of 16 k): the truncating TMEM sum of one window dominates and does not grow
// with k.  BF16 keeps 8 + 8 bits (about 4e-6 at short windows); its window error is taken as
// additive on top.
double predicted_error(int precision, int W)
{
    static const int ws[] = {1, 2, 3, 4, 5, 6, 8, 16};
    static const double es[] = {2.9e-7, 4.6e-7, 6.5e-7, 8.1e-7, 1.08e-6, 1.3e-6, 1.6e-6, 3.3e-6};
    double e = 1e-5;
    for (int i = 0; i < 8; ++i)
        if (W <= ws[i]) {
            e = es[i];
            break;
        }
    return precision == GW_PREC_BF16X3 ? 4e-6 + e : e;
}

// The longest window among 16, 8, 6, 5, 4, 3, 2, 1 chunks whose predicted error, with a quarter
// of margin, meets `target`; 0 when none does.
int window_for_target(int precision, double target)
{
    static const int cand[] = {16, 8, 6, 5, 4, 3, 2, 1};
    for (int W : cand)
        if (predicted_error(precision, W) * 1.25 <= target)
            return W;
    return 0;
}

// Upper-triangle tiles of the rank-k update (128-row blocks i of r, 256-row blocks j of r'),
// kept when the tile reaches the diagonal or above: 256 j + 255 >= 128 i.  Ordered in groups of
// 8 column blocks so that CTAs resident at the same time share operand rows in L2.
std::vector<int2> herk_tiles(int nr_pad, int bm, int bn)
{
    const int nrb = nr_pad / bm, ncb = nr_pad / bn;
    std::vector<int2> t;
    const int GROUP = 8;
    for (int j0 = 0; j0 < ncb; j0 += GROUP)
        for (int i = 0; i < nrb; ++i)
            for (int j = j0; j < std::min(ncb, j0 + GROUP); ++j)
                if (bn * j + bn - 1 >= bm * i)
                    t.push_back(make_int2(i, j));
    return t;
}

// The eps basis: integer m in FFT range with |m|^2 <= gcut, ordered by (|m|^2, m1, m2, m3).
std::vector<std::array<int, 3>> sphere_vectors(const int n[3], int gcut)
{
    std::vector<std::array<int, 4>> pts;
    for (int a = -(n[0] / 2); a < n[0] - n[0] / 2; ++a)
        for (int b = -(n[1] / 2); b < n[1] - n[1] / 2; ++b)
            for (int d = -(n[2] / 2); d < n[2] - n[2] / 2; ++d) {
                const int q = a * a + b * b + d * d;
                if (q <= gcut)
                    pts.push_back({q, a, b, d});
            }
    std::sort(pts.begin(), pts.end());
    std::vector<std::array<int, 3>> out;
    out.reserve(pts.size());
    for (auto &p : pts)
        out.push_back({p[1], p[2], p[3]});
    return out;
}

int mod(int a, int n)
{
    const int r = a % n;
    return r < 0 ? r + n : r;
}

// sqrt(V(q + G)) for the sphere in c.gvec: V = 4 pi / (Omega |q + G|^2), 0 where q + G = 0.
gw_status upload_sqrt_v(Ctx &c)
{
    const int ng = c.ng;
    std::vector<double> sv(ng, 0.0);
    const double omega = c.cell_L * c.cell_L * c.cell_L;
    const double gunit = 2.0 * PI / c.cell_L;
    for (int i = 0; i < ng; ++i) {
        const double a = c.gvec[3 * i] + c.q[0], b = c.gvec[3 * i + 1] + c.q[1], d = c.gvec[3 * i + 2] + c.q[2];
        const double m2 = a * a + b * b + d * d;  // |q + G|^2 in units of (2 pi / L)^2
        sv[i] = m2 > 0 ? std::sqrt(4.0 * PI / (omega * gunit * gunit * m2)) : 0.0;  // V(0) := 0 at q = 0
    }
    GW_TRY(ensure(c, c.d_sv, c.cap.sv, ng * sizeof(double), "sqrt(V) buffer"));
    GW_CUDA(cudaMemcpy(c.d_sv, sv.data(), ng * sizeof(double), cudaMemcpyHostToDevice), "sqrt(V) upload");
    return GW_OK;
}

gw_status build_plan(Ctx &c, int gcut)
{
    const int n[3] = {c.n1, c.n2, c.n3};
    const auto g = sphere_vectors(n, gcut);
    const int ng = static_cast<int>(g.size());
    std::vector<int> m3vals;
    for (auto &v : g)
        m3vals.push_back(v[2]);
    std::sort(m3vals.begin(), m3vals.end());
    m3vals.erase(std::unique(m3vals.begin(), m3vals.end()), m3vals.end());
    std::vector<std::array<int, 2>> dpairs;
    for (auto &v : g)
        dpairs.push_back({v[1], v[2]});
    std::sort(dpairs.begin(), dpairs.end());
    dpairs.erase(std::unique(dpairs.begin(), dpairs.end()), dpairs.end());
    const int c3 = static_cast<int>(m3vals.size()), cd = static_cast<int>(dpairs.size());

    std::vector<int> m3list(c3), disk(2 * cd), gmap(2 * ng);
    // stage-2 pairs: (m2, m3) with (-m2, m3), which share the sums over j2 and n2 - j2
    std::vector<int4> pair2;
    int k2 = 0;
    for (int d = 0; d < cd; ++d) {
        const int m2 = dpairs[d][0], m3 = dpairs[d][1];
        k2 = std::max(k2, std::abs(m2));
        if (m2 < 0)
            continue;
        const int i3 = static_cast<int>(std::lower_bound(m3vals.begin(), m3vals.end(), m3) - m3vals.begin());
        const std::array<int, 2> key = {-m2, m3};
        const auto it = std::lower_bound(dpairs.begin(), dpairs.end(), key);
        if (m2 == 0)
            pair2.push_back(make_int4(i3, 0, d, -1));
        else if (it != dpairs.end() && *it == key)
            pair2.push_back(make_int4(i3, m2, d, static_cast<int>(it - dpairs.begin())));
        else {
            pair2.clear();
            break;
        }
    }
    int covered = 0;
    for (const int4 &e : pair2)
        covered += e.w >= 0 ? 2 : 1;
    if (2 * k2 >= n[1] || covered != cd)
        pair2.clear();
    // stage-3 pairs: (m1, m2, m3) with (-m1, m2, m3), which share the sums over j1 and n1 - j1
    std::vector<int4> pair1;
    int k1 = 0;
    {
        std::vector<std::pair<std::array<int, 3>, int>> idx(ng);
        for (int i = 0; i < ng; ++i) {
            idx[i] = {g[i], i};
            k1 = std::max(k1, std::abs(g[i][0]));
        }
        std::sort(idx.begin(), idx.end());
        int cov = 0;
        for (int i = 0; i < ng && 2 * k1 < n[0]; ++i) {
            const int m1 = g[i][0];
            if (m1 < 0)
                continue;
            const int d = static_cast<int>(std::lower_bound(dpairs.begin(), dpairs.end(),
                                                            std::array<int, 2>{g[i][1], g[i][2]}) - dpairs.begin());
            if (m1 == 0) {
                pair1.push_back(make_int4(d, 0, i, -1));
                cov += 1;
                continue;
            }
            const std::pair<std::array<int, 3>, int> key = {{-m1, g[i][1], g[i][2]}, -1};
            const auto it = std::lower_bound(idx.begin(), idx.end(), key);
            if (it == idx.end() || it->first != key.first)
                break;
            pair1.push_back(make_int4(d, m1, i, it->second));
            cov += 2;
        }
        if (cov != ng)
            pair1.clear();
    }
    for (int i = 0; i < c3; ++i)
        m3list[i] = mod(m3vals[i], n[2]);
    for (int d = 0; d < cd; ++d) {
        disk[2 * d] = mod(dpairs[d][0], n[1]);
        disk[2 * d + 1] = static_cast<int>(std::lower_bound(m3vals.begin(), m3vals.end(), dpairs[d][1]) - m3vals.begin());
    }
    for (int i = 0; i < ng; ++i) {
        gmap[2 * i] = mod(g[i][0], n[0]);
        const std::array<int, 2> key = {g[i][1], g[i][2]};
        gmap[2 * i + 1] = static_cast<int>(std::lower_bound(dpairs.begin(), dpairs.end(), key) - dpairs.begin());
    }
    std::vector<float2> tw;  // exp(+2 pi i t / n_a) for the three axes, then the conjugated copy
    for (int a = 0; a < 3; ++a)
        for (int t = 0; t < n[a]; ++t) {
            const double ph = 2.0 * PI * t / n[a];
            tw.push_back(make_float2(static_cast<float>(std::cos(ph)), static_cast<float>(std::sin(ph))));
        }
    const size_t ntw = tw.size();
    for (size_t t = 0; t < ntw; ++t)
        tw.push_back(make_float2(tw[t].x, -tw[t].y));
    const size_t ints = (size_t)c3 + 2 * cd + 2 * ng;
    const size_t int_bytes = ((ints * sizeof(int) + 15) / 16) * 16;
    const size_t tw_bytes = tw.size() * sizeof(float2);
    const size_t bytes = int_bytes + tw_bytes + (pair2.size() + pair1.size()) * sizeof(int4);
    GW_TRY(ensure(c, c.d_plan_mem, c.cap.plan, bytes, "plan buffer"));
    std::vector<unsigned char> host(bytes, 0);
    std::memcpy(host.data(), m3list.data(), c3 * sizeof(int));
    std::memcpy(host.data() + c3 * sizeof(int), disk.data(), 2 * cd * sizeof(int));
    std::memcpy(host.data() + (c3 + 2 * cd) * sizeof(int), gmap.data(), 2 * ng * sizeof(int));
    std::memcpy(host.data() + int_bytes, tw.data(), tw_bytes);
    if (!pair2.empty())
        std::memcpy(host.data() + int_bytes + tw_bytes, pair2.data(), pair2.size() * sizeof(int4));
    if (!pair1.empty())
        std::memcpy(host.data() + int_bytes + tw_bytes + pair2.size() * sizeof(int4), pair1.data(),
                    pair1.size() * sizeof(int4));
    GW_CUDA(cudaMemcpy(c.d_plan_mem, host.data(), bytes, cudaMemcpyHostToDevice), "plan upload");
    DftPlan &p = c.plan;
    p.n[0] = n[0];
    p.n[1] = n[1];
    p.n[2] = n[2];
    p.ng = ng;
    p.c3 = c3;
    p.sym3 = (c3 % 2 == 1) ? (c3 - 1) / 2 : -1;
    for (int i = 0; i < c3 && p.sym3 >= 0; ++i)
        if (m3vals[i] != i - (c3 - 1) / 2)
            p.sym3 = -1;
    p.cd = cd;
    p.m3list = c.d_plan_mem;
    p.disk = c.d_plan_mem + c3;
    p.gmap = c.d_plan_mem + c3 + 2 * cd;
    p.tw = reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(c.d_plan_mem) + int_bytes);
    p.twc = p.tw + ntw;
    p.np2 = static_cast<int>(pair2.size());
    p.k2 = k2;
    p.pair2 = reinterpret_cast<int4 *>(reinterpret_cast<unsigned char *>(c.d_plan_mem) + int_bytes + tw_bytes);
    p.np1 = static_cast<int>(pair1.size());
    p.k1 = k1;
    p.pair1 = p.pair2 + pair2.size();

    c.gvec.assign(3 * ng, 0);
    for (int i = 0; i < ng; ++i) {
        c.gvec[3 * i] = g[i][0];
        c.gvec[3 * i + 1] = g[i][1];
        c.gvec[3 * i + 2] = g[i][2];
    }
    c.ng = ng;
    GW_TRY(upload_sqrt_v(c));
    // the one-kernel transform's plan, where the sphere and grid allow it
    if (c.fplan.build(n, g)) {
        GW_TRY(ensure(c, c.d_fplan, c.cap_fplan, c.fplan.device_bytes(), "transform plan"));
        GW_CUDA(c.fplan.upload(c.d_fplan, c.stream), "transform plan upload");
    }
    c.gcut = gcut;
    ++c.plan_gen;
    c.ng = ng;
    return GW_OK;
}

// eps^-1 by blocked Cholesky (eps = L L^H, Y = L^-1, eps^-1 = Y^H Y).
gw_status inverse_cholesky(Ctx &c, cudaStream_t s)
{
    const int N = c.ng, NB = CHOL_NB;
    const int nblk = (N + NB - 1) / NB;
    // workspace: A (N*N) | Y (N*N) | T (N*N) | W (N*NB) | Dinv (nblk*NB*NB)
    const size_t need = (size_t)3 * N * N + (size_t)NB * N + (size_t)nblk * NB * NB;
    GW_TRY(ensure(c, c.d_work, c.cap.work, need * sizeof(double2), "inverse workspace"));
    double2 *A = c.d_work, *Y = A + (size_t)N * N, *T = Y + (size_t)N * N, *W = T + (size_t)N * N,
            *Dinv = W + (size_t)N * NB;
    GW_CUDA(chol_inverse_enqueue(c.d_eps, N, c.d_epsinv, A, Y, T, W, Dinv, c.d_err, s), "Cholesky inverse");
    return GW_OK;
}

// eps^-1 by the Newton iteration of Sec. 5.1: X0 = eps^H / max_i sum_j |(eps eps^H)_ij|,
// X <- X (2I - eps X) until every entry moves by less than 1e-11.
gw_status inverse_newton(Ctx &c)
{
    const int N = c.ng;
    const size_t nn = (size_t)N * N;
    GW_TRY(ensure(c, c.d_work, c.cap.work, 3 * nn * sizeof(double2), "Newton workspace"));
    GW_TRY(ensure(c, c.d_scal, c.cap.scal, 4 * sizeof(double), "Newton scalars"));
    double2 *X = c.d_work, *T = X + nn, *Xn = T + nn;
    cudaStream_t s = c.stream;
    const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
    GW_CUDA(launch_zgemm(N, N, N, one, c.d_eps, N, 0, c.d_eps, N, 1, zero, T, N, s), "eps eps^H");
    GW_CUDA(launch_row_abs_sum_max(T, N, c.d_scal, s), "row sums");
    GW_CUDA(launch_scaled_adjoint(c.d_eps, N, c.d_scal, X, s), "X0");
    int it = 0;
    for (it = 1; it <= 100; ++it) {
        GW_CUDA(launch_zgemm(N, N, N, one, c.d_eps, N, 0, X, N, 0, zero, T, N, s), "eps X");
        GW_CUDA(launch_two_minus(T, N, s), "2I - eps X");
        GW_CUDA(launch_zgemm(N, N, N, one, X, N, 0, T, N, 0, zero, Xn, N, s), "X (2I - eps X)");
        GW_CUDA(launch_max_absdiff(Xn, X, nn, c.d_scal + 1, s), "max |dX|");
        double diff = 0;
        GW_CUDA(cudaMemcpyAsync(&diff, c.d_scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s), "dX readback");
        GW_CUDA(cudaStreamSynchronize(s), "Newton sync");
        std::swap(X, Xn);
        if (diff < 1e-11)
            break;
    }
    c.newton_iters = it;
    GW_CUDA(cudaMemcpyAsync(c.d_epsinv, X, nn * sizeof(double2), cudaMemcpyDeviceToDevice, s), "store eps^-1");
    return GW_OK;
}

int sm_count(int device)
{
    int nsm = 152;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        nsm = 152;
    }
    return nsm;
}

// The tensor-core Newton iteration (Sec. 5.1) for the inverse of A (n x n, device) into X.
// Kernel nodes of a captured graph: its launches, added to the launch counter on every replay.
unsigned long long kernel_nodes(cudaGraph_t g)
{
    unsigned long long k = 0;
    size_t nn = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
        std::vector<cudaGraphNode_t> nodes(nn);
        if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
            for (size_t i = 0; i < nn; ++i) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
                    ++k;
            }
    }
    cudaGetLastError();
    return k;
}

void drop_ns_graph(Ctx &c)
{
    if (c.ns_exec)
        cudaGraphExecDestroy(c.ns_exec);
    if (c.ns_graph)
        cudaGraphDestroy(c.ns_graph);
    c.ns_exec = nullptr;
    c.ns_graph = nullptr;
    c.ns_key = Ctx::NsKey{};
}

// The tensor-core Newton inverse of A (n x n) into X.  With use_graph, every step is queued in its
// graph-safe form (tables uploaded beforehand, device flags skip the unneeded steps, no host reads)
// and captured once into a CUDA graph per (n, buffers, wait limit, stream), then replayed: the
// eager form stops queuing on host reads of the convergence flag, which leave the GPU idle.
gw_status inverse_newton_tc(Ctx &c, const double2 *A, int n, double2 *X, bool use_graph = false)
{
    const int nsm = sm_count(c.device);
    GW_TRY(ensure(c, c.d_tcw, c.cap.tcw, ns_work_bytes(n, nsm), "tensor-core Newton workspace"));
    GW_TRY(ensure(c, c.d_scal, c.cap.scal, 4 * sizeof(double), "Newton scalars"));
    const uint64_t wait_ns = static_cast<uint64_t>(c.wait_limit_ms * 1e6);
    if (!use_graph) {
        // the eager form uploads the tables of order n into the workspace: a graph captured for
        // another order would then read tables of the wrong layout
        if (c.ns_exec && c.ns_key.n != n)
            drop_ns_graph(c);
        GW_CUDA(ns_inverse_enqueue(A, n, X, c.d_tcw, c.d_scal, c.d_err, wait_ns, nsm, c.stream),
                "tensor-core Newton inverse");
        return GW_OK;
    }
    Ctx::NsKey key;
    key.n = n;
    key.A = A;
    key.X = X;
    key.work = c.d_tcw;
    key.err = c.d_err;
    key.wait_ns = wait_ns;
    key.s = c.stream;
    if (!c.ns_exec || !(key == c.ns_key)) {
        drop_ns_graph(c);
        GW_CUDA(ns_prepare(c.d_tcw, n, nsm, c.stream), "Newton tables");
        // captured on a private stream (the caller's may be the legacy default stream, which
        // cannot be captured); the graph is then launched on the caller's stream
        if (!c.ns_cap_stream)
            GW_CUDA(cudaStreamCreateWithFlags(&c.ns_cap_stream, cudaStreamNonBlocking), "capture stream");
        if (cudaStreamBeginCapture(c.ns_cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, GW_E_CUDA, "stream capture of the Newton inverse could not start");
        }
        const unsigned long long counted = g_launches.load();
        // the graph queues NS_GRAPH_STEPS FP16X3 steps (every queued step costs a launch even when
        // its flag makes it return at once); an eps that needs more is finished by the eager form
        // (gw_eps_inv retries on the NS_DETAIL_CAP status)
        const cudaError_t eq = ns_inverse_enqueue(A, n, X, c.d_tcw, c.d_scal, c.d_err, wait_ns, nsm,
                                                  c.ns_cap_stream, true, NS_GRAPH_STEPS);
        g_launches.store(counted);  // captured launches run at replay time, where they are counted
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(c.ns_cap_stream, &g);
        if (eq != cudaSuccess || ec != cudaSuccess || !g) {
            cudaGetLastError();
            if (g)
                cudaGraphDestroy(g);
            return fail(c, GW_E_CUDA, "stream capture of the Newton inverse failed");
        }
        c.ns_graph = g;
        if (cudaGraphInstantiate(&c.ns_exec, c.ns_graph, 0) != cudaSuccess) {
            cudaGetLastError();
            drop_ns_graph(c);
            return fail(c, GW_E_CUDA, "instantiation of the Newton graph failed");
        }
        c.ns_graph_kernels = kernel_nodes(c.ns_graph);
        c.ns_key = key;
    }
    GW_CUDA(cudaGraphLaunch(c.ns_exec, c.stream), "Newton graph launch");
    count_launches(static_cast<int>(c.ns_graph_kernels));
    return GW_OK;
}

// Report of the last tensor-core Newton inverse of order n (after the stream has been
// synchronised): FP16X3 steps, residual after phase 1, last measured residual, refinements.
void newton_tc_record(Ctx &c, int n)
{
    double r[4] = {-1, -1, -1, -1};
    if (ns_report(c.d_tcw, n, sm_count(c.device), r) != cudaSuccess)
        cudaGetLastError();
    c.newton_iters = static_cast<int>(r[0]);
    for (int i = 0; i < 4; ++i)
        c.tc_report[i] = r[i];
}

bool is_device_pointer(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

void gw::count_launches(int n)
{
    g_launches += (unsigned long long)n;
}

void Ctx::release()
{
    dfree(d_err);
    dfree(d_psiT);
    dfree(d_E);
    dfree(d_sw);
    dfree(d_F);
    dfree(d_P);
    dfree(d_tiles);
    dfree(d_tiles_g);
    dfree(d_PG_parts);
    dfree(d_plan_mem);
    dfree(d_Q);
    dfree(d_dftw);
    dfree(d_QT);
    dfree(d_PG);
    dfree(d_sv);
    dfree(d_eps);
    dfree(d_epsinv);
    dfree(d_work);
    drop_ns_graph(*this);
    if (ns_cap_stream)
        cudaStreamDestroy(ns_cap_stream);
    ns_cap_stream = nullptr;
    dfree(d_scal);
    dfree(d_tcw);
    dfree(d_csw);
    dfree(d_Qc);
    dfree(d_fplan);
    dfree(d_cw);
    dfree(d_cgvec);
    dfree(d_cwork);
    if (h_csw)
        cudaFreeHost(h_csw);
    if (h_cw)
        cudaFreeHost(h_cw);
    h_csw = nullptr;
    h_cw = nullptr;
    if (ev_cstage)
        cudaEventDestroy(ev_cstage);
    ev_cstage = nullptr;
    dfree(d_PGsum);
    dfree(d_coef);
    dfree(d_gidx);
    dfree(d_gtw);
    dfree(d_psig);
    dfree(d_ppw);
    dfree(d_psi);
    dfree(d_psi128);
    dfree(d_small);
    for (auto &e : ev)
        if (e)
            cudaEventDestroy(e);
}

extern "C" {

const char *gw_status_str(int st)
{
    switch (st) {
    case GW_OK: return "ok";
    case GW_E_INVALID: return "invalid argument";
    case GW_E_NOMEM: return "out of device memory";
    case GW_E_CUDA: return "CUDA error";
    case GW_E_NOT_READY: return "call-order violation";
    case GW_E_NUMERIC: return "eps not positive definite";
    case GW_E_TIMEOUT: return "device wait ran out";
    case GW_E_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
    }
}

int gw_version(void)
{
    return 1;
}

gw_status gw_create(gw_ctx **out, int device, void *stream)
{
    if (!out)
        return GW_E_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return GW_E_INVALID;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess)
        return GW_E_CUDA;
    if (prop.major != 10 || prop.minor != 3)
        return GW_E_UNSUPPORTED;  // the kernels are built for sm_103a only
    gw_ctx *h = new (std::nothrow) gw_ctx;
    if (!h)
        return GW_E_NOMEM;
    Ctx &c = h->c;
    c.device = device;
    c.stream = static_cast<cudaStream_t>(stream);
    if (cudaSetDevice(device) != cudaSuccess || cudaMalloc(&c.d_err, sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(c.d_err, 0, sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        c.release();
        delete h;
        return GW_E_CUDA;
    }
    for (auto &e : c.ev)
        cudaEventCreate(&e);
    *out = h;
    return GW_OK;
}

gw_status gw_destroy(gw_ctx *h)
{
    if (!h)
        return GW_E_INVALID;
    cudaSetDevice(h->c.device);
    cudaStreamSynchronize(h->c.stream);
    h->c.release();
    delete h;
    return GW_OK;
}

gw_status gw_set_stream(gw_ctx *h, void *stream)
{
    if (!h)
        return GW_E_INVALID;
    h->c.stream = static_cast<cudaStream_t>(stream);
    return GW_OK;
}

gw_status gw_last_error(const gw_ctx *h, char *buf, size_t n)
{
    if (!h || !buf || n == 0)
        return GW_E_INVALID;
    std::snprintf(buf, n, "%s", h->c.last_error.c_str());
    return GW_OK;
}

gw_status gw_set_wait_limit(gw_ctx *h, double ms)
{
    if (!h || !(ms > 0.0) || ms > 600000.0)
        return GW_E_INVALID;
    h->c.wait_limit_ms = ms;
    return GW_OK;
}

gw_status gw_set_q(gw_ctx *h, const double *q)
{
    if (!h || !q || !std::isfinite(q[0]) || !std::isfinite(q[1]) || !std::isfinite(q[2]))
        return GW_E_INVALID;
    Ctx &c = h->c;
    for (int a = 0; a < 3; ++a)
        c.q[a] = q[a];
    c.eps_ready = false;
    if (c.ng > 0 && c.gcut >= 0) {  // a sphere exists: the next gw_eps_inv uses V(q + G)
        GW_CUDA(cudaSetDevice(c.device), "set device");
        GW_CUDA(cudaStreamSynchronize(c.stream), "sync before sqrt(V) update");
        GW_TRY(upload_sqrt_v(c));
    }
    return GW_OK;
}

gw_status gw_set_herk_window(gw_ctx *h, int window_chunks, int flush_windows)
{
    if (!h || window_chunks < 1 || window_chunks > 64 || flush_windows < 1 || flush_windows > 4096)
        return GW_E_INVALID;
    h->c.herk_W = window_chunks;
    h->c.herk_L = flush_windows;
    h->c.err_target = 0.0;
    return GW_OK;
}

gw_status gw_set_herk_kernel(gw_ctx *h, int kind)
{
    if (!h || (kind != GW_HERK_SINGLE && kind != GW_HERK_PAIR))
        return GW_E_INVALID;
    h->c.herk_kernel = kind;
    return GW_OK;
}

gw_status gw_set_error_target(gw_ctx *h, double target)
{
    if (!h || !(target >= 0.0) || !std::isfinite(target))
        return GW_E_INVALID;
    if (target > 0.0 && window_for_target(GW_PREC_FP16X3, target) == 0)
        return fail(h->c, GW_E_UNSUPPORTED, "no window length meets the error target %g", target);
    h->c.err_target = target;
    return GW_OK;
}

gw_status gw_set_timing(gw_ctx *h, int enable)
{
    if (!h)
        return GW_E_INVALID;
    h->c.timing = enable != 0;
    return GW_OK;
}

gw_status gw_get_times(gw_ctx *h, float *t6)
{
    if (!h || !t6)
        return GW_E_INVALID;
    Ctx &c = h->c;
    GW_CUDA(cudaStreamSynchronize(c.stream), "timing sync");
    resolve_times(c);
    for (int i = 0; i < 6; ++i)
        t6[i] = c.times[i];
    return GW_OK;
}

gw_status gw_get_stats(gw_ctx *h, double *s8)
{
    if (!h || !s8)
        return GW_E_INVALID;
    Ctx &c = h->c;
    GW_CUDA(cudaStreamSynchronize(c.stream), "stats sync");
    resolve_times(c);
    s8[0] = (double)g_launches.load();
    s8[1] = c.newton_iters;
    s8[2] = c.times_n[1] ? c.times_sum[1] / c.times_n[1] : 0.0;
    s8[3] = c.times_n[1];
    int e = 0;
    if (c.d_small && (c.F_prec == GW_PREC_FP16X3 || c.F_prec == GW_PREC_BF16X3))
        cudaMemcpy(&e, c.d_small + 1, sizeof(int), cudaMemcpyDeviceToHost);
    s8[4] = e;
    s8[5] = c.n_tiles;
    s8[6] = c.last_W;
    s8[7] = c.herk_L;
    return GW_OK;
}

gw_status gw_reset_times(gw_ctx *h)
{
    if (!h)
        return GW_E_INVALID;
    for (int i = 0; i < 6; ++i) {
        h->c.times_sum[i] = 0.0;
        h->c.times_n[i] = 0;
    }
    return GW_OK;
}

gw_status gw_load_states(gw_ctx *h, int n1, int n2, int n3, double cell_L, int nv, int nc, const void *psi,
                         int psi_dtype, int psi_on_device, const double *energies_eV)
{
    if (!h)
        return GW_E_INVALID;
    Ctx &c = h->c;
    if (n1 < 2 || n2 < 2 || n3 < 2 || n1 > 64 || n2 > 64 || n3 > 64)
        return fail(c, GW_E_INVALID, "grid %d x %d x %d outside [2, 64]^3", n1, n2, n3);
    const int nr = n1 * n2 * n3;
    if (nv < 1 || nc < 1 || (long long)nv + nc > nr)
        return fail(c, GW_E_INVALID, "need nv, nc >= 1 and nv + nc <= N_r (got %d, %d, %d)", nv, nc, nr);
    if ((long long)nv * nc > (1LL << 30))
        return fail(c, GW_E_INVALID, "nv * nc too large");
    if (!(cell_L > 0.0) || !std::isfinite(cell_L))
        return fail(c, GW_E_INVALID, "cell_L must be positive and finite");
    if (!psi || !energies_eV)
        return fail(c, GW_E_INVALID, "null psi or energies");
    if (psi_dtype != GW_C64 && psi_dtype != GW_C128)
        return fail(c, GW_E_INVALID, "psi_dtype must be GW_C64 or GW_C128");
    const int nb = nv + nc;
    double emax_v = -INFINITY, emin_c = INFINITY;
    std::vector<double> Eh(nb);
    for (int i = 0; i < nb; ++i) {
        if (!std::isfinite(energies_eV[i]))
            return fail(c, GW_E_INVALID, "energy %d is not finite", i);
        Eh[i] = energies_eV[i] / HARTREE_EV;
        if (i < nv)
            emax_v = std::max(emax_v, energies_eV[i]);
        else
            emin_c = std::min(emin_c, energies_eV[i]);
    }
    if (!(emax_v < emin_c))
        return fail(c, GW_E_INVALID, "need max(E_v) < min(E_c) (got %g >= %g eV)", emax_v, emin_c);
    if (psi_on_device && !is_device_pointer(psi))
        return fail(c, GW_E_INVALID, "psi_on_device set but psi is not a device pointer");

    GW_CUDA(cudaSetDevice(c.device), "set device");
    c.loaded = c.P_ready = c.PG_ready = c.eps_ready = false;
    c.q_pairs = false;
    c.n1 = n1;
    c.n2 = n2;
    c.n3 = n3;
    c.nr = nr;
    c.nv = nv;
    c.nc = nc;
    c.nb = nb;
    c.cell_L = cell_L;
    c.k = nv * nc;
    c.kpad = ((c.k + HERK_KC - 1) / HERK_KC) * HERK_KC;
    c.sw_max = static_cast<float>(std::sqrt(2.0 / ((emin_c - emax_v) / HARTREE_EV)));
    c.nr_pad = ((nr + HERK_BN - 1) / HERK_BN) * HERK_BN;
    c.gcut = -1;
    c.ng = 0;
    const size_t n = (size_t)nb * nr;
    cudaStream_t s = c.stream;
    GW_TRY(ensure(c, c.d_psiT, c.cap.psiT, n * sizeof(float2), "transposed states"));
    GW_TRY(ensure(c, c.d_E, c.cap.E, nb * sizeof(double), "energies"));
    GW_TRY(ensure(c, c.d_sw, c.cap.sw, (size_t)c.k * sizeof(float), "weights"));
    const float2 *src = nullptr;
    if (psi_dtype == GW_C64 && psi_on_device) {
        src = static_cast<const float2 *>(psi);
    } else {
        GW_TRY(ensure(c, c.d_psi, c.cap.psi, n * sizeof(float2), "state staging"));
        if (psi_dtype == GW_C64) {
            GW_CUDA(cudaMemcpyAsync(c.d_psi, psi, n * sizeof(float2), cudaMemcpyHostToDevice, s), "copy states");
        } else {
            const double2 *p128 = static_cast<const double2 *>(psi);
            if (!psi_on_device) {
                GW_TRY(ensure(c, c.d_psi128, c.cap.psi128, n * sizeof(double2), "complex128 staging"));
                GW_CUDA(cudaMemcpyAsync(c.d_psi128, psi, n * sizeof(double2), cudaMemcpyHostToDevice, s),
                        "copy states");
                p128 = c.d_psi128;
            }
            GW_CUDA(launch_c128_to_c64(p128, n, c.d_psi, s), "round states");
        }
        src = c.d_psi;
    }
    GW_CUDA(launch_check_finite(src, n, c.d_err, s), "check states");
    GW_CUDA(launch_transpose_states(src, nb, nr, c.d_psiT, s), "transpose states");
    GW_CUDA(cudaMemcpyAsync(c.d_E, Eh.data(), nb * sizeof(double), cudaMemcpyHostToDevice, s), "copy energies");
    GW_CUDA(launch_weights(c.d_E, nv, nc, c.d_sw, s), "weights");
    // Eh is a local: make sure the copy has consumed it before returning.
    GW_CUDA(cudaStreamSynchronize(s), "load sync");
    c.E_h = Eh;
    c.loaded = true;
    return GW_OK;
}

gw_status gw_build_P(gw_ctx *h, int precision, void *P_out)
{
    if (!h)
        return GW_E_INVALID;
    Ctx &c = h->c;
    if (!c.loaded)
        return fail(c, GW_E_NOT_READY, "gw_build_P before gw_load_states");
    if (precision != GW_PREC_TF32X3 && precision != GW_PREC_TF32X1 && precision != GW_PREC_FP32_SIMT &&
        precision != GW_PREC_FP16X3 && precision != GW_PREC_BF16X3)
        return fail(c, GW_E_INVALID, "unknown precision %d", precision);
    GW_CUDA(cudaSetDevice(c.device), "set device");
    cudaStream_t s = c.stream;
    const bool p16 = precision == GW_PREC_FP16X3 || precision == GW_PREC_BF16X3;
    if (p16) {
        c.last_W = c.err_target > 0.0 ? window_for_target(precision, c.err_target) : c.herk_W;
        if (c.last_W == 0)
            return fail(c, GW_E_UNSUPPORTED, "no window length meets the error target %g at this precision",
                        c.err_target);
    }
    const int kchunk = p16 ? HERK16_KC : HERK_KC;
    c.kpad = ((c.k + kchunk - 1) / kchunk) * kchunk;
    // CTA pairs take 256-row blocks of r: nr_pad is a multiple of 256 for every grid
    const bool pair = p16 && c.herk_kernel == GW_HERK_PAIR && c.nr_pad % 256 == 0;
    const int npl = pair ? HERK16_NPL_PAIR : HERK16_NPL;
    size_t Fbytes;
    if (precision == GW_PREC_FP32_SIMT)
        Fbytes = (size_t)c.kpad * c.nr_pad * sizeof(float2);
    else if (p16)
        Fbytes = (size_t)c.kpad * c.nr_pad * 2 * npl;
    else
        Fbytes = (size_t)c.kpad * c.nr_pad * sizeof(float) * (precision == GW_PREC_TF32X3 ? 4 : 2);
    GW_TRY(ensure(c, c.d_F, c.cap.F, Fbytes, "pair-density operand"));
    if (!c.d_small)
        GW_CUDA(cudaMalloc(&c.d_small, 4 * sizeof(unsigned)), "scale words");
    c.F_bytes = Fbytes;
    c.P_bytes = (size_t)c.nr * c.nr * sizeof(float2);
    GW_TRY(ensure(c, c.d_P, c.cap.P, c.P_bytes, "P(r,r')"));
    c.P_ready = c.PG_ready = c.eps_ready = false;

    const int tile_kind = pair ? 2 : p16 ? 1 : 0;
    if (precision != GW_PREC_FP32_SIMT && (c.tiles_nr_pad != c.nr_pad || c.tiles_kind != tile_kind)) {
        const auto t = pair  ? herk_pair_tiles(c.nr_pad)
                       : p16 ? herk_tiles(c.nr_pad, HERK16_T, HERK16_T)
                             : herk_tiles(c.nr_pad, HERK_BM, HERK_BN);
        GW_TRY(ensure(c, c.d_tiles, c.cap.tiles, t.size() * sizeof(int2), "tile list"));
        GW_CUDA(cudaMemcpy(c.d_tiles, t.data(), t.size() * sizeof(int2), cudaMemcpyHostToDevice), "tile upload");
        c.n_tiles = static_cast<int>(t.size());
        c.tiles_nr_pad = c.nr_pad;
        c.tiles_kind = tile_kind;
    }
    const uint64_t wait_ns = static_cast<uint64_t>(c.wait_limit_ms * 1e6);
    int *scale_exp = reinterpret_cast<int *>(c.d_small + 1);

    record(c, 0);
    if (p16)
        GW_CUDA(launch_pair_density16(c.d_psiT, c.d_sw, c.sw_max, c.nr, c.nb, c.nv, c.nc, c.kpad, c.nr_pad,
                                      precision == GW_PREC_BF16X3, c.d_small, scale_exp,
                                      reinterpret_cast<uint16_t *>(c.d_F), s, npl),
                "pair densities (16-bit)");
    else
        GW_CUDA(launch_pair_density(c.d_psiT, c.d_sw, c.nr, c.nb, c.nv, c.nc, c.kpad, c.nr_pad, precision, c.d_F, s),
                "pair densities");
    c.F_prec = precision;
    if (p16)
        c.last_herk_kernel = pair ? GW_HERK_PAIR : GW_HERK_SINGLE;
    record(c, 1);
    if (precision == GW_PREC_FP32_SIMT) {
        GW_CUDA(launch_herk_simt(reinterpret_cast<float2 *>(c.d_F), c.kpad, c.nr, c.nr_pad, c.d_P, s),
                "rank-k update (CUDA cores)");
    } else if (pair) {
        GW_CUDA(launch_herk16x2(reinterpret_cast<uint16_t *>(c.d_F), precision == GW_PREC_BF16X3, c.kpad, c.nr,
                                c.nr_pad, c.d_tiles, c.n_tiles, c.d_P, scale_exp, c.d_err, wait_ns, c.last_W,
                                c.herk_L, s),
                "rank-k update (tcgen05 CTA pairs, 16-bit)");
    } else if (p16) {
        GW_CUDA(launch_herk16(reinterpret_cast<uint16_t *>(c.d_F), precision == GW_PREC_BF16X3, c.kpad, c.nr,
                              c.nr_pad, c.d_tiles, c.n_tiles, c.d_P, scale_exp, c.d_err, wait_ns, c.last_W, c.herk_L,
                              s),
                "rank-k update (tcgen05, 16-bit)");
    } else {
        GW_CUDA(launch_herk_tc(c.d_F, precision, c.kpad, c.nr, c.nr_pad, c.d_tiles, c.n_tiles, c.d_P, c.d_err, wait_ns,
                               s),
                "rank-k update (tcgen05, TF32)");
    }
    record(c, 2);
    if (P_out)
        GW_CUDA(cudaMemcpyAsync(P_out, c.d_P, c.P_bytes, cudaMemcpyDefault, s), "copy P out");
    c.P_ready = true;
    return GW_OK;
}

// The k-point weight and running sum (gw_set_kweight) applied to the P~ just formed in d_PG.
gw_status finish_PG(Ctx &c, cudaStream_t s)
{
    const int ng = c.ng;
    const size_t n = (size_t)ng * ng;
    if (c.kaccumulate && c.PGsum_ng != ng)
        return fail(c, c.PGsum_ng < 0 ? GW_E_NOT_READY : GW_E_INVALID,
                    "k-point accumulation needs an earlier P~ on the same sphere (N_g %d, sum has %d)", ng,
                    c.PGsum_ng);
    if (c.kaccumulate || c.kweight != 1.0)
        GW_CUDA(launch_kweight(c.d_PG, c.d_PGsum, n, static_cast<float>(c.kweight), c.kaccumulate, s), "k weight");
    GW_TRY(ensure(c, c.d_PGsum, c.cap.PGsum, n * sizeof(float2), "P~ sum over k"));
    GW_CUDA(cudaMemcpyAsync(c.d_PGsum, c.d_PG, n * sizeof(float2), cudaMemcpyDeviceToDevice, s), "keep P~ sum");
    c.PGsum_ng = ng;
    return GW_OK;
}

// Sphere transform of rows of X: the one-kernel form where the plan and the alignment allow it
// (and the context has not asked for the two-kernel form), else the two-kernel form.  With sw set,
// the rows are the pair densities conj(psi_v) psi_c sw[k] of the states X = psi (c from state c0).
cudaError_t transform_rows(Ctx &c, const float2 *X, long long ldx, int rows, float2 *Y, long long ldy, bool negexp,
                           cudaStream_t s, const float *sw = nullptr, int nv = 0, int nc = 1, int c0 = -1)
{
    if (c.transform_kind == GW_TRANSFORM_FUSED && c.fplan.ok) {
        const uint64_t wait_ns = static_cast<uint64_t>(c.wait_limit_ms * 1e6);
        const cudaError_t e = launch_dft_fused(X, ldx, rows, Y, ldy, c.fplan, negexp, sw, nv, nc, c0 < 0 ? nv : c0,
                                               c.d_err, wait_ns, s);
        if (e != cudaErrorNotSupported)
            return e;
    }
    const bool cst = c.transform_kind != GW_TRANSFORM_TABLES;
    if (sw)
        return launch_dft_pairs_ws(X, ldx, sw, nv, nc, Y, ldy, c.plan, c.d_dftw, s, negexp, c0, cst);
    return launch_dft_rows_ws(X, ldx, rows, Y, ldy, c.plan, c.d_dftw, s, negexp, cst);
}

gw_status gw_set_transform_kernel(gw_ctx *h, int kind)
{
    if (!h || (kind != GW_TRANSFORM_TWO_KERNEL && kind != GW_TRANSFORM_FUSED && kind != GW_TRANSFORM_TABLES))
        return GW_E_INVALID;
    h->c.transform_kind = kind;
    return GW_OK;
}

gw_status gw_P_to_G(gw_ctx *h, int gcut, int *ng_out, int *gvec_out, int max_ng, void *PG_out)
{
    if (!h)
        return GW_E_INVALID;
    Ctx &c = h->c;
    if (!c.P_ready)
        return fail(c, GW_E_NOT_READY, "gw_P_to_G before gw_build_P");
    const int nmin = std::min(c.n1, std::min(c.n2, c.n3));
    if (gcut < 0 || 4LL * gcut >= (long long)nmin * nmin)
        return fail(c, GW_E_INVALID, "gcut %d must satisfy 0 <= 4 gcut < min(n)^2 = %d", gcut, nmin * nmin);
    GW_CUDA(cudaSetDevice(c.device), "set device");
    if (gcut != c.gcut)
        GW_TRY(build_plan(c, gcut));
    const int ng = c.ng;
    if (gvec_out && ng > max_ng)
        return fail(c, GW_E_INVALID, "N_g = %d exceeds max_ng = %d", ng, max_ng);
    if (!dft_supported(c.plan))
        return fail(c, GW_E_UNSUPPORTED, "sphere too large for the transform kernel (N_g = %d)", ng);
    cudaStream_t s = c.stream;
    GW_TRY(ensure(c, c.d_Q, c.cap.Q, (size_t)c.nr * ng * sizeof(float2), "row transform"));
    c.q_pairs = false;
    GW_TRY(ensure(c, c.d_QT, c.cap.QT, (size_t)c.nr * ng * sizeof(float2), "transposed row transform"));
    GW_TRY(ensure(c, c.d_PG, c.cap.PG, (size_t)ng * ng * sizeof(float2), "P~"));
    GW_TRY(ensure(c, c.d_dftw, c.cap.dftw, dft_work_bytes(c.plan, std::max(c.nr, ng)), "transform workspace"));
    c.PG_ready = c.eps_ready = false;
    record(c, 3);
    // Q[r'][G] = sum_r P[r'][r] e^{+iG.r} = conj(P^(G, r')) since P is Hermitian
    GW_CUDA(transform_rows(c, c.d_P, c.nr, c.nr, c.d_Q, ng, false, s), "row transform");
    record(c, 4);
    // QT[G][r'] = conj(Q[r'][G]) = P^(G, r');  P~[G][G'] = sum_r' QT[G][r'] e^{+iG'.r'}
    GW_CUDA(launch_conj_transpose(c.d_Q, c.nr, ng, c.d_QT, s), "conjugate transpose");
    GW_CUDA(transform_rows(c, c.d_QT, c.nr, ng, c.d_PG, ng, false, s), "column transform");
    GW_CUDA(launch_hermitize(c.d_PG, ng, s), "Hermitian part of P~");
    GW_TRY(finish_PG(c, s));
    record(c, 5);
    if (PG_out)
        GW_CUDA(cudaMemcpyAsync(PG_out, c.d_PG, (size_t)ng * ng * sizeof(float2), cudaMemcpyDefault, s),
                "copy P~ out");
    if (ng_out)
        *ng_out = ng;
    if (gvec_out)
        std::memcpy(gvec_out, c.gvec.data(), (size_t)3 * ng * sizeof(int));
    c.PG_ready = true;
    return GW_OK;
}

// P~ by the g-space route (Eq. gpsaceP): M_k(G) = sum_r exp(-iG.r) f_k(r) for every pair density
// f_k, then P~(G, G') = -sum_k M_k(G) conj(M_k(G')) as a rank-k update of N_g x N_g.  P(r,r') is
// never formed.
gw_status gw_build_PG(gw_ctx *h, int precision, int gcut, int *ng_out, int *gvec_out, int max_ng, void *PG_out)
{
    if (!h)
        return GW_E_INVALID;
    Ctx &c = h->c;
    if (!c.loaded)
        return fail(c, GW_E_NOT_READY, "gw_build_PG before gw_load_states");
    if (precision != GW_PREC_FP16X3 && precision != GW_PREC_BF16X3)
        return fail(c, GW_E_INVALID, "gw_build_PG takes GW_PREC_FP16X3 or GW_PREC_BF16X3, not %d", precision);
    const int nmin = std::min(c.n1, std::min(c.n2, c.n3));
    if (gcut < 0 || 4LL * gcut >= (long long)nmin * nmin)
        return fail(c, GW_E_INVALID, "gcut %d must satisfy 0 <= 4 gcut < min(n)^2 = %d", gcut, nmin * nmin);
    GW_CUDA(cudaSetDevice(c.device), "set device");
    if (gcut != c.gcut)
        GW_TRY(build_plan(c, gcut));
    const int ng = c.ng;
    if (gvec_out && ng > max_ng)
        return fail(c, GW_E_INVALID, "N_g = %d exceeds max_ng = %d", ng, max_ng);
    if (!dft_supported(c.plan))
        return fail(c, GW_E_UNSUPPORTED, "sphere too large for the transform kernel (N_g = %d)", ng);
    cudaStream_t s = c.stream;
    const bool bf16 = precision == GW_PREC_BF16X3;
    c.last_W = c.err_target > 0.0 ? window_for_target(precision, c.err_target) : c.herk_W;
    if (c.last_W == 0)
        return fail(c, GW_E_UNSUPPORTED, "no window length meets the error target %g at this precision",
                    c.err_target);
    const int k = c.k, kpad = ((k + HERK16_KC - 1) / HERK16_KC) * HERK16_KC;
    const int ng_pad = ((ng + 255) / 256) * 256;
    // buffers: the pair-density transforms [k][ng] in Q, the 16-bit planes of the transforms in QT,
    // the result in PG (pair densities [k][nr_pad] complex64 in F only where the transform kernel
    // cannot form them itself)
    GW_TRY(ensure(c, c.d_Q, c.cap.Q, (size_t)k * ng * sizeof(float2), "pair-density transforms"));
    GW_TRY(ensure(c, c.d_QT, c.cap.QT, (size_t)kpad * ng_pad * 2 * HERK16_NPL, "transform planes"));
    GW_TRY(ensure(c, c.d_PG, c.cap.PG, (size_t)ng * ng * sizeof(float2), "P~"));
    GW_TRY(ensure(c, c.d_dftw, c.cap.dftw, dft_work_bytes(c.plan, k), "transform workspace"));
    if (!c.d_small)
        GW_CUDA(cudaMalloc(&c.d_small, 4 * sizeof(unsigned)), "scale words");
    if (c.tiles_g_pad != ng_pad) {
        const auto t = herk_tiles(ng_pad, HERK16_T, HERK16_T);
        GW_TRY(ensure(c, c.d_tiles_g, c.cap.tiles_g, t.size() * sizeof(int2), "tile list (N_g)"));
        GW_CUDA(cudaMemcpy(c.d_tiles_g, t.data(), t.size() * sizeof(int2), cudaMemcpyHostToDevice), "tile upload");
        c.n_tiles_g = static_cast<int>(t.size());
        c.tiles_g_pad = ng_pad;
    }
    c.F_prec = -1;  // F no longer holds the operand of gw_build_P (nor its scale word)
    c.P_ready = c.PG_ready = c.eps_ready = false;
    const uint64_t wait_ns = static_cast<uint64_t>(c.wait_limit_ms * 1e6);
    int *scale_exp = reinterpret_cast<int *>(c.d_small + 1);

    record(c, 0);
    // The states back in [nb][N_r] order (psiT transposed), so that the transform kernel forms
    // each pair density from two contiguous state lines; grids that need the row-block kernel
    // store the pair densities first.
    GW_TRY(ensure(c, c.d_psi, c.cap.psi, (size_t)c.nb * c.nr * sizeof(float2), "state staging"));
    GW_CUDA(launch_transpose_states(c.d_psiT, c.nr, c.nb, c.d_psi, s), "states [nb][N_r]");
    record(c, 1);
    record(c, 3);
    c.q_pairs = false;
    cudaError_t fe = transform_rows(c, c.d_psi, c.nr, k, c.d_Q, ng, true, s, c.d_sw, c.nv, c.nc);
    if (fe == cudaErrorNotSupported) {
        GW_TRY(ensure(c, c.d_F, c.cap.F, (size_t)k * c.nr_pad * sizeof(float2), "pair densities"));
        float2 *Fc = reinterpret_cast<float2 *>(c.d_F);
        GW_CUDA(launch_pair_density_rows(c.d_psiT, c.d_sw, c.nr, c.nb, c.nv, c.nc, k, c.nr_pad, Fc, s),
                "pair densities");
        fe = launch_dft_rows_ws(Fc, c.nr_pad, k, c.d_Q, ng, c.plan, c.d_dftw, s, true,
                                c.transform_kind != GW_TRANSFORM_TABLES);
    }
    GW_CUDA(fe, "pair-density transforms");
    c.q_pairs = true;  // the closure estimate may reuse them (gw_corr_closure)
    c.q_pairs_gen = c.plan_gen;
    record(c, 4);
    GW_CUDA(launch_planes16_from_c64(c.d_Q, k, ng, ng, kpad, ng_pad, bf16, c.d_small, scale_exp,
                                     reinterpret_cast<uint16_t *>(c.d_QT), s),
            "transform planes");
    // one CTA per SM: split k so that tiles x splits fills the GPU
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c.device);
    const int splits = std::max(1, std::min(kpad / HERK16_KC, nsm / std::max(1, c.n_tiles_g)));
    if (splits > 1)
        GW_TRY(ensure(c, c.d_PG_parts, c.cap.PG_parts, (size_t)splits * ng * ng * sizeof(float2), "split-k partials"));
    GW_CUDA(launch_herk16(reinterpret_cast<const uint16_t *>(c.d_QT), bf16, kpad, ng, ng_pad, c.d_tiles_g,
                          c.n_tiles_g, c.d_PG, scale_exp, c.d_err, wait_ns, c.last_W, c.herk_L, s, splits,
                          c.d_PG_parts),
            "rank-k update in G space");
    GW_TRY(finish_PG(c, s));
    record(c, 5);
    if (PG_out)
        GW_CUDA(cudaMemcpyAsync(PG_out, c.d_PG, (size_t)ng * ng * sizeof(float2), cudaMemcpyDefault, s),
                "copy P~ out");
    if (ng_out)
        *ng_out = ng;
    if (gvec_out)
        std::memcpy(gvec_out, c.gvec.data(), (size_t)3 * ng * sizeof(int));
    c.PG_ready = true;
    return GW_OK;
}

gw_status gw_corr_closure(gw_ctx *h, int gcut, const double *E_omit_eV, int nc_omit, void *out)
{
    if (!h)
        return GW_E_INVALID;
    Ctx &c = h->c;
    if (!c.loaded)
        return fail(c, GW_E_NOT_READY, "gw_corr_closure before gw_load_states");
    if (!out || nc_omit < 0 || (nc_omit > 0 && !E_omit_eV))
        return fail(c, GW_E_INVALID, "null output or omitted energies, or nc_omit < 0");
    if (!is_device_pointer(out))
        return fail(c, GW_E_INVALID, "the closure estimate is written to device memory");
    if (c.nr <= c.nb)
        return fail(c, GW_E_INVALID, "the loaded states already span the grid (N_r = %d, %d states)", c.nr, c.nb);
    const int nmin = std::min(c.n1, std::min(c.n2, c.n3));
    if (gcut < 0 || 4LL * gcut >= (long long)nmin * nmin)
        return fail(c, GW_E_INVALID, "gcut %d must satisfy 0 <= 4 gcut < min(n)^2 = %d", gcut, nmin * nmin);
    // W_v = sum over the omitted c of 2 / (E_v - E_c) (Hartree, FP64), divided by N_r - n_in
    const double inv_dim = 1.0 / (double)(c.nr - c.nb);
    std::vector<double> wv(c.nv, 0.0);
    for (int i = 0; i < nc_omit; ++i) {
        const double eo = E_omit_eV[i] / HARTREE_EV;
        if (!std::isfinite(eo))
            return fail(c, GW_E_INVALID, "omitted energy %d is not finite", i);
        for (int v = 0; v < c.nv; ++v) {
            if (!(eo > c.E_h[v]))
                return fail(c, GW_E_INVALID, "omitted energy %d is not above occupied energy %d", i, v);
            wv[v] += 2.0 / (c.E_h[v] - eo);
        }
    }
    // pair weights sqrt(-W_v / (N_r - n_in)): [nv][nb] for every loaded n, then [nv][nv] for the
    // occupied n alone (the rows added to gw_build_PG's transforms when those are reused)
    std::vector<float> csw((size_t)c.nv * c.nb + (size_t)c.nv * c.nv);
    for (int v = 0; v < c.nv; ++v) {
        wv[v] *= inv_dim;
        const float x = static_cast<float>(std::sqrt(-wv[v]));
        for (int n = 0; n < c.nb; ++n)
            csw[(size_t)v * c.nb + n] = x;
        for (int n = 0; n < c.nv; ++n)
            csw[(size_t)c.nv * c.nb + (size_t)v * c.nv + n] = x;
    }
    GW_CUDA(cudaSetDevice(c.device), "set device");
    if (gcut != c.gcut)
        GW_TRY(build_plan(c, gcut));
    const int ng = c.ng;
    if (!dft_supported(c.plan))
        return fail(c, GW_E_UNSUPPORTED, "sphere too large for the transform kernel (N_g = %d)", ng);
    cudaStream_t s = c.stream;
    const int k2 = c.nv * c.nb, kpad2 = ((k2 + HERK16_KC - 1) / HERK16_KC) * HERK16_KC;
    const int ng_pad = ((ng + 255) / 256) * 256;
    // gw_build_PG on the same states and sphere left the transforms M_vc(G) sqrt(2/(E_c - E_v)) of
    // the unoccupied pairs in Q: rescaled, they are nv nc of the k2 rows, and only the nv nv occupied
    // pairs are transformed here
    const bool reuse = c.q_pairs && c.q_pairs_gen == c.plan_gen && c.nc > 0;
    GW_TRY(ensure(c, c.d_csw, c.cap_csw, csw.size() * sizeof(float), "closure weights"));
    GW_TRY(ensure(c, c.d_cw, c.cap_cw, wv.size() * sizeof(double), "closure state weights"));
    GW_TRY(ensure(c, c.d_cgvec, c.cap_cgvec, (size_t)3 * ng * sizeof(int), "closure sphere"));
    GW_TRY(ensure(c, c.d_cwork, c.cap_cwork, closure_work_bytes(c.nr), "closure workspace"));
    if (reuse)
        GW_TRY(ensure(c, c.d_Qc, c.cap_Qc, (size_t)k2 * ng * sizeof(float2), "closure matrix elements"));
    else
        GW_TRY(ensure(c, c.d_Q, c.cap.Q, (size_t)k2 * ng * sizeof(float2), "closure matrix elements"));
    float2 *Qk = reuse ? c.d_Qc : c.d_Q;
    GW_TRY(ensure(c, c.d_QT, c.cap.QT, (size_t)kpad2 * ng_pad * 2 * HERK16_NPL, "closure planes"));
    GW_TRY(ensure(c, c.d_dftw, c.cap.dftw, dft_work_bytes(c.plan, k2), "transform workspace"));
    GW_TRY(ensure(c, c.d_psi, c.cap.psi, (size_t)c.nb * c.nr * sizeof(float2), "state staging"));
    if (!c.d_small)
        GW_CUDA(cudaMalloc(&c.d_small, 4 * sizeof(unsigned)), "scale words");
    if (c.tiles_g_pad != ng_pad) {
        const auto t = herk_tiles(ng_pad, HERK16_T, HERK16_T);
        GW_TRY(ensure(c, c.d_tiles_g, c.cap.tiles_g, t.size() * sizeof(int2), "tile list (N_g)"));
        GW_CUDA(cudaMemcpy(c.d_tiles_g, t.data(), t.size() * sizeof(int2), cudaMemcpyHostToDevice), "tile upload");
        c.n_tiles_g = static_cast<int>(t.size());
        c.tiles_g_pad = ng_pad;
    }
    c.F_prec = -1;  // the scale word now belongs to the closure's planes
    // the weights through pinned staging: wait for the previous call's upload to have read it
    if (c.cstage_pending) {
        GW_CUDA(cudaEventSynchronize(c.ev_cstage), "closure staging");
        c.cstage_pending = false;
    }
    if (!c.ev_cstage)
        GW_CUDA(cudaEventCreateWithFlags(&c.ev_cstage, cudaEventDisableTiming), "closure staging event");
    if (c.cap_hcsw < csw.size()) {
        if (c.h_csw)
            cudaFreeHost(c.h_csw);
        c.h_csw = nullptr;
        c.cap_hcsw = 0;
        GW_CUDA(cudaMallocHost(&c.h_csw, csw.size() * sizeof(float)), "closure staging");
        c.cap_hcsw = csw.size();
    }
    if (c.cap_hcw < wv.size()) {
        if (c.h_cw)
            cudaFreeHost(c.h_cw);
        c.h_cw = nullptr;
        c.cap_hcw = 0;
        GW_CUDA(cudaMallocHost(&c.h_cw, wv.size() * sizeof(double)), "closure staging");
        c.cap_hcw = wv.size();
    }
    std::copy(csw.begin(), csw.end(), c.h_csw);
    std::copy(wv.begin(), wv.end(), c.h_cw);
    GW_CUDA(cudaMemcpyAsync(c.d_csw, c.h_csw, csw.size() * sizeof(float), cudaMemcpyHostToDevice, s),
            "closure weights");
    GW_CUDA(cudaMemcpyAsync(c.d_cw, c.h_cw, wv.size() * sizeof(double), cudaMemcpyHostToDevice, s),
            "closure state weights");
    GW_CUDA(cudaEventRecord(c.ev_cstage, s), "closure staging event");
    c.cstage_pending = true;
    // the sphere vectors once per plan, the twiddles once per grid (both synchronous, both rare)
    if (c.cgvec_buf != c.d_cgvec || c.cgvec_gen != c.plan_gen) {
        GW_CUDA(cudaMemcpyAsync(c.d_cgvec, c.gvec.data(), (size_t)3 * ng * sizeof(int), cudaMemcpyHostToDevice, s),
                "closure sphere");
        GW_CUDA(cudaStreamSynchronize(s), "closure sphere");
        c.cgvec_buf = c.d_cgvec;
        c.cgvec_gen = c.plan_gen;
    }
    {
        const int dims[3] = {c.n1, c.n2, c.n3};
        if (c.ctw_buf != c.d_cwork || c.ctw_dims[0] != dims[0] || c.ctw_dims[1] != dims[1] ||
            c.ctw_dims[2] != dims[2]) {
            GW_CUDA(closure_set_twiddles(dims, c.nr, c.d_cwork, s), "closure twiddles");
            c.ctw_buf = c.d_cwork;
            for (int a = 0; a < 3; ++a)
                c.ctw_dims[a] = dims[a];
        }
    }
    const uint64_t wait_ns = static_cast<uint64_t>(c.wait_limit_ms * 1e6);
    int *scale_exp = reinterpret_cast<int *>(c.d_small + 1);
    float2 *o = static_cast<float2 *>(out);
    // projector term: matrix elements M_vn(G) sqrt(-W_v / (N_r - n_in)) for every loaded n, then the
    // N_g x N_g rank-k update (which returns minus the sum of the outer products) into `out`
    GW_CUDA(launch_transpose_states(c.d_psiT, c.nr, c.nb, c.d_psi, s), "states [nb][N_r]");
    cudaError_t fe;
    if (reuse) {
        const int kv = c.nv * c.nc;
        GW_CUDA(launch_closure_rescale(c.d_Q, c.nv, c.nc, ng, c.d_csw, c.nb, c.d_sw, c.d_Qc, s),
                "closure matrix elements from the pair transforms");
        fe = transform_rows(c, c.d_psi, c.nr, c.nv * c.nv, c.d_Qc + (size_t)kv * ng, ng, true, s,
                            c.d_csw + (size_t)c.nv * c.nb, c.nv, c.nv, 0);
    } else {
        c.q_pairs = false;
        fe = transform_rows(c, c.d_psi, c.nr, k2, c.d_Q, ng, true, s, c.d_csw, c.nv, c.nb, 0);
    }
    if (fe == cudaErrorNotSupported)
        return fail(c, GW_E_UNSUPPORTED, "the closure needs the plane transform kernel for this grid");
    GW_CUDA(fe, "closure matrix elements");
    GW_CUDA(launch_planes16_from_c64(Qk, k2, ng, ng, kpad2, ng_pad, false, c.d_small, scale_exp,
                                     reinterpret_cast<uint16_t *>(c.d_QT), s),
            "closure planes");
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c.device);
    const int splits = std::max(1, std::min(kpad2 / HERK16_KC, nsm / std::max(1, c.n_tiles_g)));
    if (splits > 1)
        GW_TRY(ensure(c, c.d_PG_parts, c.cap.PG_parts, (size_t)splits * ng * ng * sizeof(float2), "split-k partials"));
    GW_CUDA(launch_herk16(reinterpret_cast<const uint16_t *>(c.d_QT), false, kpad2, ng, ng_pad, c.d_tiles_g,
                          c.n_tiles_g, o, scale_exp, c.d_err, wait_ns, c.herk_W, c.herk_L, s, splits, c.d_PG_parts),
            "closure projector term");
    // density term rho_W(G - G') / (N_r - n_in), combined in place with the projector term
    const int dims[3] = {c.n1, c.n2, c.n3};
    GW_CUDA(closure_enqueue(c.d_psiT, c.nr, c.nb, c.nv, c.d_cw, dims, c.d_cgvec, ng, o, o, c.d_cwork, s),
            "closure density term");
    return GW_OK;
}

gw_status gw_eps_inv(gw_ctx *h, int method, void *eps_out, void *epsinv_out)
{
    if (!h)
        return GW_E_INVALID;
    Ctx &c = h->c;
    if (!c.PG_ready)
        return fail(c, GW_E_NOT_READY, "gw_eps_inv before gw_P_to_G");
    if (method != GW_INV_CHOLESKY && method != GW_INV_NEWTON && method != GW_INV_NEWTON_TC)
        return fail(c, GW_E_INVALID, "unknown inversion method %d", method);
    GW_CUDA(cudaSetDevice(c.device), "set device");
    // the call reads the device status back (a stream synchronisation), which a stream under
    // capture does not allow: refuse before anything is queued into the caller's capture
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c.stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return fail(c, GW_E_INVALID, "gw_eps_inv synchronises its stream, which is being captured");
    }
    const int ng = c.ng;
    const size_t bytes = (size_t)ng * ng * sizeof(double2);
    GW_TRY(ensure(c, c.d_eps, c.cap.eps, bytes, "eps"));
    GW_TRY(ensure(c, c.d_epsinv, c.cap.epsinv, bytes, "eps^-1"));
    cudaStream_t s = c.stream;
    record(c, 6);
    GW_CUDA(launch_eps_build(c.d_PG, c.d_sv, ng, c.d_eps, s), "eps build");
    record(c, 7);
    if (method == GW_INV_CHOLESKY)
        GW_TRY(inverse_cholesky(c, c.stream));
    else if (method == GW_INV_NEWTON)
        GW_TRY(inverse_newton(c));
    else
        GW_TRY(inverse_newton_tc(c, c.d_eps, ng, c.d_epsinv, true));
    record(c, 8);
    if (eps_out)
        GW_CUDA(cudaMemcpyAsync(eps_out, c.d_eps, bytes, cudaMemcpyDefault, s), "copy eps out");
    if (epsinv_out)
        GW_CUDA(cudaMemcpyAsync(epsinv_out, c.d_epsinv, bytes, cudaMemcpyDefault, s), "copy eps^-1 out");
    gw_status st = read_device_status(c);
    if (st == GW_E_NUMERIC && method == GW_INV_NEWTON_TC && ((c.last_status >> 8) & 0xFFu) == SITE_NS &&
        (c.last_status >> 16) == NS_DETAIL_CAP) {
        // the graph's FP16X3 steps were too few for this eps: the eager form runs up to 16, each
        // stopping test on the host
        GW_TRY(inverse_newton_tc(c, c.d_eps, ng, c.d_epsinv, false));
        if (eps_out)
            GW_CUDA(cudaMemcpyAsync(eps_out, c.d_eps, bytes, cudaMemcpyDefault, s), "copy eps out");
        if (epsinv_out)
            GW_CUDA(cudaMemcpyAsync(epsinv_out, c.d_epsinv, bytes, cudaMemcpyDefault, s), "copy eps^-1 out");
        st = read_device_status(c);
    }
    resolve_times(c);
    if (method == GW_INV_NEWTON_TC)
        newton_tc_record(c, ng);
    c.eps_ready = st == GW_OK;
    return st;
}

gw_status gw_set_kweight(gw_ctx *h, double weight, int accumulate)
{
    if (!h)
        return GW_E_INVALID;
    Ctx &c = h->c;
    if (!std::isfinite(weight))
        return fail(c, GW_E_INVALID, "k-point weight must be finite");
    c.kweight = weight;
    c.kaccumulate = accumulate != 0;
    return GW_OK;
}

gw_status gw_load_states_g(gw_ctx *h, int n1, int n2, int n3, double cell_L, int nv, int nc, int npw,
                           const int *gvec_psi, const void *coef, int coef_dtype, int coef_on_device,
                           const double *energies_eV)
{
    if (!h)
        return GW_E_INVALID;
    Ctx &c = h->c;
    if (n1 < 2 || n2 < 2 || n3 < 2 || n1 > 64 || n2 > 64 || n3 > 64)
        return fail(c, GW_E_INVALID, "grid %d x %d x %d outside [2, 64]^3", n1, n2, n3);
    const int nr = n1 * n2 * n3;
    const int nb = nv + nc;
    if (nv < 1 || nc < 1 || (long long)nv + nc > nr)
        return fail(c, GW_E_INVALID, "need nv, nc >= 1 and nv + nc <= N_r (got %d, %d, %d)", nv, nc, nr);
    if (npw < 1 || npw > nr)
        return fail(c, GW_E_INVALID, "npw = %d plane waves: need 1 <= npw <= N_r = %d", npw, nr);
    if (!gvec_psi || !coef || !energies_eV)
        return fail(c, GW_E_INVALID, "null gvec, coefficients or energies");
    if (coef_dtype != GW_C64 && coef_dtype != GW_C128)
        return fail(c, GW_E_INVALID, "coef_dtype must be GW_C64 or GW_C128");
    if (coef_on_device && !is_device_pointer(coef))
        return fail(c, GW_E_INVALID, "coef_on_device set but coef is not a device pointer");
    // Miller indices modulo the grid; two plane waves on one grid point would alias
    std::vector<int> idx(npw);
    std::vector<char> seen(nr, 0);
    const int nn[3] = {n1, n2, n3};
    for (int p = 0; p < npw; ++p) {
        int j[3];
        for (int a = 0; a < 3; ++a)
            j[a] = ((gvec_psi[3 * p + a] % nn[a]) + nn[a]) % nn[a];
        const int lin = (j[0] * n2 + j[1]) * n3 + j[2];
        if (seen[lin])
            return fail(c, GW_E_INVALID, "plane wave %d (%d, %d, %d) aliases an earlier one on the %d x %d x %d grid",
                        p, gvec_psi[3 * p], gvec_psi[3 * p + 1], gvec_psi[3 * p + 2], n1, n2, n3);
        seen[lin] = 1;
        idx[p] = lin;
    }
    std::vector<float2> tw(n1 + n2 + n3);
    for (int a = 0, o = 0; a < 3; o += nn[a], ++a)
        for (int t = 0; t < nn[a]; ++t) {
            const double ph = 6.283185307179586476925 * t / nn[a];
            tw[o + t] = make_float2(static_cast<float>(std::cos(ph)), static_cast<float>(std::sin(ph)));
        }
    GW_CUDA(cudaSetDevice(c.device), "set device");
    cudaStream_t s = c.stream;
    const size_t ncoef = (size_t)nb * npw, n = (size_t)nb * nr;
    GW_TRY(ensure(c, c.d_gidx, c.cap.gidx, npw * sizeof(int), "plane-wave indices"));
    GW_TRY(ensure(c, c.d_gtw, c.cap.gtw, tw.size() * sizeof(float2), "axis twiddles"));
    GW_TRY(ensure(c, c.d_psig, c.cap.psig, n * sizeof(float2), "state transform workspace"));
    GW_TRY(ensure(c, c.d_psi, c.cap.psi, n * sizeof(float2), "state staging"));
    GW_CUDA(cudaMemcpyAsync(c.d_gidx, idx.data(), npw * sizeof(int), cudaMemcpyHostToDevice, s), "copy indices");
    GW_CUDA(cudaMemcpyAsync(c.d_gtw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, s),
            "copy twiddles");
    const float2 *coef64 = nullptr;
    if (coef_dtype == GW_C64 && coef_on_device) {
        coef64 = static_cast<const float2 *>(coef);
    } else {
        GW_TRY(ensure(c, c.d_coef, c.cap.coef, ncoef * sizeof(float2), "coefficient staging"));
        if (coef_dtype == GW_C64) {
            GW_CUDA(cudaMemcpyAsync(c.d_coef, coef, ncoef * sizeof(float2), cudaMemcpyHostToDevice, s),
                    "copy coefficients");
        } else {
            const double2 *p128 = static_cast<const double2 *>(coef);
            if (!coef_on_device) {
                GW_TRY(ensure(c, c.d_psi128, c.cap.psi128, ncoef * sizeof(double2), "complex128 staging"));
                GW_CUDA(cudaMemcpyAsync(c.d_psi128, coef, ncoef * sizeof(double2), cudaMemcpyHostToDevice, s),
                        "copy coefficients");
                p128 = c.d_psi128;
            }
            GW_CUDA(launch_c128_to_c64(p128, ncoef, c.d_coef, s), "round coefficients");
        }
        coef64 = c.d_coef;
    }
    GW_CUDA(launch_states_from_g(coef64, nb, npw, c.d_gidx, n1, n2, n3, c.d_gtw, c.d_psig, c.d_psi, s),
            "states to the grid");
    // host vectors idx and tw are read by the copies above: finish them before they go out of scope
    GW_CUDA(cudaStreamSynchronize(s), "transform sync");
    return gw_load_states(h, n1, n2, n3, cell_L, nv, nc, c.d_psi, GW_C64, 1, energies_eV);
}

gw_status gw_pp_modes(gw_ctx *h, int nmodes, double tol, double *sigma, double *omega2, double *resid, void *A_out)
{
    if (!h)
        return GW_E_INVALID;
    Ctx &c = h->c;
    if (!c.eps_ready || !c.loaded)
        return fail(c, GW_E_NOT_READY, "gw_pp_modes needs gw_eps_inv (and the states it came from)");
    const int ng = c.ng;
    int b = std::min(40, std::max(2 * nmodes + 8, 16));
    b = std::min(b, ng - (ng & 1));  // even, at most N_g
    if (nmodes < 1 || nmodes > 16 || nmodes > b)
        return fail(c, GW_E_INVALID, "nmodes %d: need 1 <= nmodes <= min(16, N_g) (N_g = %d)", nmodes, ng);
    if (!(tol > 0.0) || !std::isfinite(tol))
        return fail(c, GW_E_INVALID, "tol must be positive");
    GW_CUDA(cudaSetDevice(c.device), "set device");
    cudaStream_t s = c.stream;
    c.pp_ready = false;
    const size_t bytes = PPWork::carve(nullptr, ng, b, c.nr).bytes;
    GW_TRY(ensure(c, c.d_ppw, c.cap.ppw, bytes, "plasmon-pole workspace"));
    c.pp = PPWork::carve(c.d_ppw, ng, b, c.nr);
    const int dims[3] = {c.n1, c.n2, c.n3};
    std::vector<int> g32(c.gvec.begin(), c.gvec.end());
    GW_CUDA(pp_prepare(c.pp, c.d_epsinv, c.d_sv, c.d_psiT, ng, c.nr, c.nb, c.nv, dims, g32.data(), c.cell_L, c.q, s),
            "plasmon-pole S, density and Omega");
    int iters = 0;
    GW_CUDA(pp_iterate(c.pp, ng, b, nmodes, tol, 400, &iters, s), "plasmon-pole subspace iteration");
    std::vector<double> th(b), res(b), w2(b);
    int flag = 0;
    GW_CUDA(cudaMemcpyAsync(th.data(), c.pp.theta, b * sizeof(double), cudaMemcpyDeviceToHost, s), "read theta");
    GW_CUDA(cudaMemcpyAsync(res.data(), c.pp.res, b * sizeof(double), cudaMemcpyDeviceToHost, s), "read residuals");
    GW_CUDA(cudaMemcpyAsync(w2.data(), c.pp.omega2, b * sizeof(double), cudaMemcpyDeviceToHost, s), "read omega2");
    GW_CUDA(cudaMemcpyAsync(&flag, c.pp.flag, sizeof(int), cudaMemcpyDeviceToHost, s), "read flag");
    if (A_out)
        GW_CUDA(cudaMemcpy2DAsync(A_out, nmodes * sizeof(double2), c.pp.X, b * sizeof(double2),
                                  nmodes * sizeof(double2), ng, cudaMemcpyDefault, s),
                "copy modes out");
    GW_TRY(read_device_status(c));
    for (int a = 0; a < nmodes; ++a) {
        if (sigma)
            sigma[a] = th[a];
        if (omega2)
            omega2[a] = w2[a];
        if (resid)
            resid[a] = res[a];
    }
    bool conv = flag == 0;
    for (int a = 0; a < nmodes; ++a)
        conv = conv && res[a] <= tol * std::fabs(th[0]);
    if (!conv)
        return fail(c, GW_E_NUMERIC, "plasmon-pole modes did not converge in %d iterations (residual %g)", iters,
                    res[0]);
    c.pp_b = b;
    c.pp_nmodes = nmodes;
    c.pp_ready = true;
    return GW_OK;
}

gw_status gw_pp_eval(gw_ctx *h, double omega, int nuse, void *S_out)
{
    if (!h)
        return GW_E_INVALID;
    Ctx &c = h->c;
    if (!c.pp_ready)
        return fail(c, GW_E_NOT_READY, "gw_pp_eval before gw_pp_modes");
    if (nuse < 1 || nuse > c.pp_nmodes || !S_out || !std::isfinite(omega))
        return fail(c, GW_E_INVALID, "gw_pp_eval: nuse %d (1..%d), finite omega, non-null output", nuse,
                    c.pp_nmodes);
    GW_CUDA(cudaSetDevice(c.device), "set device");
    cudaStream_t s = c.stream;
    const int ng = c.ng;
    GW_CUDA(pp_eval(c.pp, ng, c.pp_b, nuse, omega, c.pp.Om, s), "S(omega)");
    GW_CUDA(cudaMemcpyAsync(S_out, c.pp.Om, (size_t)ng * ng * sizeof(double2), cudaMemcpyDefault, s), "copy S out");
    return read_device_status(c);
}

gw_status gw_zgemm_tc(gw_ctx *h, int mode, int M, int N, int K, const void *A, int lda, const void *B, int ldb,
                      void *C)
{
    if (!h)
        return GW_E_INVALID;
    Ctx &c = h->c;
    if (mode != 0 && mode != 1)
        return fail(c, GW_E_INVALID, "gw_zgemm_tc: mode %d (0 = FP16X3, 1 = integer slices)", mode);
    if (M < 1 || N < 1 || K < 1 || M > 16384 || N > 16384 || K > 16384 || lda < K || ldb < N)
        return fail(c, GW_E_INVALID, "gw_zgemm_tc: sizes M %d N %d K %d lda %d ldb %d", M, N, K, lda, ldb);
    if (!A || !B || !C || !is_device_pointer(A) || !is_device_pointer(B) || !is_device_pointer(C))
        return fail(c, GW_E_INVALID, "gw_zgemm_tc: A, B and C must be device pointers");
    GW_CUDA(cudaSetDevice(c.device), "set device");
    ZPlan p;
    p.build(mode, M, N, K, sm_count(c.device));
    GW_TRY(ensure(c, c.d_tcw, c.cap.tcw, zgemm_work_bytes(p), "zgemm workspace"));
    const uint64_t wait_ns = static_cast<uint64_t>(c.wait_limit_ms * 1e6);
    GW_CUDA(zgemm_enqueue(p, static_cast<const double2 *>(A), lda, static_cast<const double2 *>(B), ldb,
                          static_cast<double2 *>(C), c.d_tcw, c.d_err, wait_ns, c.stream),
            "tensor-core zgemm");
    return read_device_status(c);
}

gw_status gw_zinv_tc(gw_ctx *h, int n, const void *A, void *X)
{
    if (!h)
        return GW_E_INVALID;
    Ctx &c = h->c;
    if (n < 1 || n > 16384)
        return fail(c, GW_E_INVALID, "gw_zinv_tc: order %d", n);
    if (!A || !X || !is_device_pointer(A) || !is_device_pointer(X))
        return fail(c, GW_E_INVALID, "gw_zinv_tc: A and X must be device pointers");
    GW_CUDA(cudaSetDevice(c.device), "set device");
    GW_TRY(inverse_newton_tc(c, static_cast<const double2 *>(A), n, static_cast<double2 *>(X)));
    const gw_status st = read_device_status(c);
    newton_tc_record(c, n);
    return st;
}

gw_status gw_newton_tc_report(gw_ctx *h, double *out4)
{
    if (!h || !out4)
        return GW_E_INVALID;
    for (int i = 0; i < 4; ++i)
        out4[i] = h->c.tc_report[i];
    return GW_OK;
}

gw_status gw_sync(gw_ctx *h)
{
    if (!h)
        return GW_E_INVALID;
    return read_device_status(h->c);
}

gw_status gw_get_buffer(gw_ctx *h, int which, void **ptr, size_t *bytes)
{
    if (!h || !ptr || !bytes)
        return GW_E_INVALID;
    Ctx &c = h->c;
    *ptr = nullptr;
    *bytes = 0;
    switch (which) {
    case GW_BUF_P:
        if (!c.P_ready)
            return GW_E_NOT_READY;
        *ptr = c.d_P;
        *bytes = c.P_bytes;
        return GW_OK;
    case GW_BUF_F:
        if (c.F_prec < 0 || !c.P_ready)
            return GW_E_NOT_READY;
        *ptr = c.d_F;
        *bytes = c.F_bytes;
        return GW_OK;
    case GW_BUF_PG:
        if (!c.PG_ready)
            return GW_E_NOT_READY;
        *ptr = c.d_PG;
        *bytes = (size_t)c.ng * c.ng * sizeof(float2);
        return GW_OK;
    case GW_BUF_EPS:
    case GW_BUF_EPSINV:
        if (!c.eps_ready)
            return GW_E_NOT_READY;
        *ptr = which == GW_BUF_EPS ? (void *)c.d_eps : (void *)c.d_epsinv;
        *bytes = (size_t)c.ng * c.ng * sizeof(double2);
        return GW_OK;
    case GW_BUF_WEIGHTS:
        if (!c.loaded)
            return GW_E_NOT_READY;
        *ptr = c.d_sw;
        *bytes = (size_t)c.k * sizeof(float);
        return GW_OK;
    case GW_BUF_PSIT:
        if (!c.loaded)
            return GW_E_NOT_READY;
        *ptr = c.d_psiT;
        *bytes = (size_t)c.nr * c.nb * sizeof(float2);
        return GW_OK;
    default:
        return GW_E_INVALID;
    }
}

gw_status gw_get_dims(gw_ctx *h, int *d)
{
    if (!h || !d)
        return GW_E_INVALID;
    Ctx &c = h->c;
    if (!c.loaded)
        return GW_E_NOT_READY;
    d[0] = c.n1;
    d[1] = c.n2;
    d[2] = c.n3;
    d[3] = c.nr;
    d[4] = c.nv;
    d[5] = c.nc;
    d[6] = c.PG_ready ? c.ng : 0;
    d[7] = c.nr_pad;
    return GW_OK;
}

}  // extern "C"

// ============================================================================= batch
// Independent systems of uneven size (q-points, supercells) in one pass: per-instance pair
// densities, ONE persistent launch of the rank-k update over every instance's tiles, then each
// instance's transforms, eps and FP64 inverse.  The whole pass can be captured once in a CUDA
// graph and replayed.  Every instance keeps its own context (buffers, status word, results).

struct gw_batch {
    std::vector<gw_ctx *> ctxs;
    std::vector<int> gcut;
    int precision = GW_PREC_FP16X3;
    int device = 0;
    cudaStream_t stream = nullptr;  // the batch's own non-blocking stream
    bool own_stream = false;
    HerkJob *d_jobs = nullptr;
    int4 *d_tiles = nullptr;
    int n_tiles = 0, grid = 0;
    int W = 2, L = 256;
    uint32_t *d_err = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float herk_ms = 0.f;
    int runs = 0;
    int graph_kernels = 0;          // kernel nodes of the captured pass (launches per replay)
    int inv_method = GW_INV_NEWTON_TC;  // eps^-1 of every instance (gw_batch_set_inverse)
    std::string last_error;
};

namespace {

gw_status vbfail(gw_batch &b, gw_status st, const char *fmt, va_list ap)
{
    char buf[512];
    vsnprintf(buf, sizeof buf, fmt, ap);
    b.last_error = buf;
    return st;
}

gw_status bfail(gw_batch &b, gw_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    const gw_status r = vbfail(b, st, fmt, ap);
    va_end(ap);
    return r;
}

gw_status bfail(gw_batch *b, gw_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    const gw_status r = vbfail(*b, st, fmt, ap);
    va_end(ap);
    return r;
}

#define GW_BCUDA(call, where)                                                                  \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            cudaGetLastError();                                                                \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? GW_E_NOMEM : GW_E_CUDA, "%s: %s", \
                         where, cudaGetErrorString(e_));                                       \
        }                                                                                      \
    } while (0)

void drop_graph(gw_batch &b)
{
    if (b.exec)
        cudaGraphExecDestroy(b.exec);
    if (b.graph)
        cudaGraphDestroy(b.graph);
    b.exec = nullptr;
    b.graph = nullptr;
}

// Allocate every buffer the pass needs (graph capture must not allocate) and build the plans.
gw_status batch_prepare(gw_batch &b)
{
    const bool bf16 = b.precision == GW_PREC_BF16X3;
    std::vector<HerkJob> jobs;
    std::vector<int4> tiles;
    for (size_t i = 0; i < b.ctxs.size(); ++i) {
        Ctx &c = b.ctxs[i]->c;
        const int kpad = ((c.k + HERK16_KC - 1) / HERK16_KC) * HERK16_KC;
        c.kpad = kpad;
        const size_t Fbytes = (size_t)kpad * c.nr_pad * 2 * HERK16_NPL;
        GW_TRY(ensure(c, c.d_F, c.cap.F, Fbytes, "pair-density operand"));
        if (!c.d_small)
            GW_CUDA(cudaMalloc(&c.d_small, 4 * sizeof(unsigned)), "scale words");
        c.F_bytes = Fbytes;
        c.P_bytes = (size_t)c.nr * c.nr * sizeof(float2);
        GW_TRY(ensure(c, c.d_P, c.cap.P, c.P_bytes, "P(r,r')"));
        if (b.gcut[i] != c.gcut)
            GW_TRY(build_plan(c, b.gcut[i]));
        if (!dft_supported(c.plan))
            return fail(c, GW_E_UNSUPPORTED, "sphere too large for the transform kernel (N_g = %d)", c.ng);
        const int ng = c.ng, NB = CHOL_NB, nblk = (ng + NB - 1) / NB;
        GW_TRY(ensure(c, c.d_Q, c.cap.Q, (size_t)c.nr * ng * sizeof(float2), "row transform"));
        c.q_pairs = false;
        GW_TRY(ensure(c, c.d_QT, c.cap.QT, (size_t)c.nr * ng * sizeof(float2), "transposed row transform"));
        GW_TRY(ensure(c, c.d_PG, c.cap.PG, (size_t)ng * ng * sizeof(float2), "P~"));
        GW_TRY(ensure(c, c.d_dftw, c.cap.dftw, dft_work_bytes(c.plan, std::max(c.nr, ng)), "transform workspace"));
        GW_TRY(ensure(c, c.d_eps, c.cap.eps, (size_t)ng * ng * sizeof(double2), "eps"));
        GW_TRY(ensure(c, c.d_epsinv, c.cap.epsinv, (size_t)ng * ng * sizeof(double2), "eps^-1"));
        if (b.inv_method == GW_INV_NEWTON_TC) {
            const int nsm = sm_count(c.device);
            GW_TRY(ensure(c, c.d_tcw, c.cap.tcw, ns_work_bytes(ng, nsm), "tensor-core Newton workspace"));
            GW_TRY(ensure(c, c.d_scal, c.cap.scal, 4 * sizeof(double), "Newton scalars"));
            GW_CUDA(ns_prepare(c.d_tcw, ng, nsm, b.stream), "Newton tables");
        } else {
            const size_t work = (size_t)3 * ng * ng + (size_t)NB * ng + (size_t)nblk * NB * NB;
            GW_TRY(ensure(c, c.d_work, c.cap.work, work * sizeof(double2), "inverse workspace"));
        }
        jobs.push_back({reinterpret_cast<const uint16_t *>(c.d_F), c.d_P, reinterpret_cast<const int *>(c.d_small + 1),
                        c.nr, c.nr_pad, kpad, 0});
        for (const int2 t : herk_tiles(c.nr_pad, HERK16_T, HERK16_T))
            tiles.push_back(make_int4((int)i, t.x, t.y, 0));
    }
    // longest tiles first: with the static round-robin schedule every CTA gets a similar load
    std::stable_sort(tiles.begin(), tiles.end(),
                     [&](const int4 &a, const int4 &c2) { return jobs[a.x].kpad > jobs[c2.x].kpad; });
    if (b.d_jobs)
        cudaFree(b.d_jobs);
    if (b.d_tiles)
        cudaFree(b.d_tiles);
    b.d_jobs = nullptr;
    b.d_tiles = nullptr;
    GW_BCUDA(cudaMalloc(&b.d_jobs, jobs.size() * sizeof(HerkJob)), "job table");
    GW_BCUDA(cudaMalloc(&b.d_tiles, tiles.size() * sizeof(int4)), "tile table");
    GW_BCUDA(cudaMemcpy(b.d_jobs, jobs.data(), jobs.size() * sizeof(HerkJob), cudaMemcpyHostToDevice), "job upload");
    GW_BCUDA(cudaMemcpy(b.d_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice), "tile upload");
    b.n_tiles = static_cast<int>(tiles.size());
    int sms = 0;
    GW_BCUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b.device), "SM count");
    b.grid = std::min(b.n_tiles, sms);
    (void)bf16;
    return GW_OK;
}

gw_status batch_pair_densities(gw_batch &b)
{
    for (gw_ctx *h : b.ctxs) {
        Ctx &c = h->c;
        GW_CUDA(launch_pair_density16(c.d_psiT, c.d_sw, c.sw_max, c.nr, c.nb, c.nv, c.nc, c.kpad, c.nr_pad,
                                      b.precision == GW_PREC_BF16X3, c.d_small, reinterpret_cast<int *>(c.d_small + 1),
                                      reinterpret_cast<uint16_t *>(c.d_F), b.stream),
                "pair densities (batch)");
        c.F_prec = b.precision;
    }
    return GW_OK;
}

gw_status batch_herk(gw_batch &b)
{
    const uint64_t wait_ns = static_cast<uint64_t>(b.ctxs[0]->c.wait_limit_ms * 1e6);
    GW_BCUDA(cudaEventRecord(b.e0, b.stream), "event");
    GW_BCUDA(launch_herk16p(b.d_jobs, b.d_tiles, b.n_tiles, b.grid, b.precision == GW_PREC_BF16X3, b.d_err, wait_ns,
                            b.W, b.L, b.stream),
             "rank-k update (persistent, batch)");
    GW_BCUDA(cudaEventRecord(b.e1, b.stream), "event");
    return GW_OK;
}

// The whole pass, launches only (no allocation, no host synchronisation): safe to capture.
gw_status batch_enqueue(gw_batch &b)
{
    GW_TRY(batch_pair_densities(b));
    GW_TRY(batch_herk(b));
    for (gw_ctx *h : b.ctxs) {
        Ctx &c = h->c;
        const int ng = c.ng;
        cudaStream_t s = b.stream;
        GW_CUDA(transform_rows(c, c.d_P, c.nr, c.nr, c.d_Q, ng, false, s), "row transform");
        GW_CUDA(launch_conj_transpose(c.d_Q, c.nr, ng, c.d_QT, s), "conjugate transpose");
        GW_CUDA(transform_rows(c, c.d_QT, c.nr, ng, c.d_PG, ng, false, s), "column transform");
        GW_CUDA(launch_hermitize(c.d_PG, ng, s), "Hermitian part of P~");
        GW_CUDA(launch_eps_build(c.d_PG, c.d_sv, ng, c.d_eps, s), "eps build");
        if (b.inv_method == GW_INV_NEWTON_TC) {
            const uint64_t wait_ns = static_cast<uint64_t>(c.wait_limit_ms * 1e6);
            GW_CUDA(ns_inverse_enqueue(c.d_eps, ng, c.d_epsinv, c.d_tcw, c.d_scal, c.d_err, wait_ns,
                                       sm_count(c.device), s, true),
                    "tensor-core Newton inverse");
        } else {
            GW_TRY(inverse_cholesky(c, s));
        }
    }
    return GW_OK;
}

gw_status batch_status(gw_batch &b)
{
    GW_BCUDA(cudaStreamSynchronize(b.stream), "batch synchronize");
    uint32_t word = 0;
    GW_BCUDA(cudaMemcpy(&word, b.d_err, sizeof word, cudaMemcpyDeviceToHost), "status readback");
    if (word != 0) {
        cudaMemset(b.d_err, 0, sizeof(uint32_t));
        return bfail(b, static_cast<gw_status>(word & 0xFF), "rank-k update: device wait ran out (block %u)",
                     word >> 16);
    }
    gw_status first = GW_OK;
    for (gw_ctx *h : b.ctxs) {
        Ctx &c = h->c;
        const gw_status st = read_device_status(c);
        c.P_ready = c.PG_ready = c.eps_ready = st == GW_OK;
        if (st != GW_OK && first == GW_OK) {
            first = st;
            b.last_error = c.last_error;
        }
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b.e0, b.e1) == cudaSuccess)
        b.herk_ms = ms;
    cudaGetLastError();
    return first;
}

std::string batch_key(const gw_batch &b)
{
    std::string k = "prec" + std::to_string(b.precision);
    for (size_t i = 0; i < b.ctxs.size(); ++i) {
        const Ctx &c = b.ctxs[i]->c;
        k += "|" + std::to_string(c.n1) + "x" + std::to_string(c.n2) + "x" + std::to_string(c.n3) + ",v" +
             std::to_string(c.nv) + ",c" + std::to_string(c.nc) + ",g" + std::to_string(b.gcut[i]);
    }
    return k;
}

}  // namespace

extern "C" {

gw_status gw_batch_create(gw_batch **out, gw_ctx *const *ctxs, int n, const int *gcuts, int precision)
{
    if (!out || !ctxs || !gcuts || n < 1 || n > 4096)
        return GW_E_INVALID;
    *out = nullptr;
    if (precision != GW_PREC_FP16X3 && precision != GW_PREC_BF16X3)
        return GW_E_UNSUPPORTED;
    gw_batch *b = new (std::nothrow) gw_batch;
    if (!b)
        return GW_E_NOMEM;
    b->precision = precision;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || !ctxs[i]->c.loaded) {
            delete b;
            return GW_E_NOT_READY;
        }
        const Ctx &c = ctxs[i]->c;
        const int nmin = std::min(c.n1, std::min(c.n2, c.n3));
        if (i > 0 && (c.device != ctxs[0]->c.device || c.stream != ctxs[0]->c.stream)) {
            delete b;
            return GW_E_INVALID;  // one device and one stream for the whole batch
        }
        if (gcuts[i] < 0 || 4LL * gcuts[i] >= (long long)nmin * nmin) {
            delete b;
            return GW_E_INVALID;
        }
        b->ctxs.push_back(ctxs[i]);
        b->gcut.push_back(gcuts[i]);
    }
    b->device = ctxs[0]->c.device;
    // the pass runs on a stream of its own: the contexts' stream may be the legacy default
    // stream, which cannot be captured into a graph
    if (cudaSetDevice(b->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return GW_E_CUDA;
    }
    b->own_stream = true;
    if (cudaSetDevice(b->device) != cudaSuccess || cudaMalloc(&b->d_err, sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(b->d_err, 0, sizeof(uint32_t)) != cudaSuccess || cudaEventCreate(&b->e0) != cudaSuccess ||
        cudaEventCreate(&b->e1) != cudaSuccess) {
        cudaGetLastError();
        gw_batch_destroy(b);
        return GW_E_CUDA;
    }
    const gw_status st = batch_prepare(*b);
    if (st != GW_OK) {
        gw_batch_destroy(b);
        return st;
    }
    *out = b;
    return GW_OK;
}

gw_status gw_batch_destroy(gw_batch *b)
{
    if (!b)
        return GW_E_INVALID;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    drop_graph(*b);
    if (b->d_jobs)
        cudaFree(b->d_jobs);
    if (b->d_tiles)
        cudaFree(b->d_tiles);
    if (b->d_err)
        cudaFree(b->d_err);
    if (b->e0)
        cudaEventDestroy(b->e0);
    if (b->e1)
        cudaEventDestroy(b->e1);
    if (b->own_stream && b->stream)
        cudaStreamDestroy(b->stream);
    delete b;
    return GW_OK;
}

gw_status gw_batch_set_window(gw_batch *b, int window_chunks, int flush_windows)
{
    if (!b || window_chunks < 1 || window_chunks > 64 || flush_windows < 1 || flush_windows > 4096)
        return GW_E_INVALID;
    if (b->W != window_chunks || b->L != flush_windows)
        drop_graph(*b);  // the captured launch carries the old lengths
    b->W = window_chunks;
    b->L = flush_windows;
    return GW_OK;
}

gw_status gw_batch_set_inverse(gw_batch *b, int method)
{
    if (!b || (method != GW_INV_CHOLESKY && method != GW_INV_NEWTON_TC))
        return GW_E_INVALID;
    if (b->inv_method == method)
        return GW_OK;
    drop_graph(*b);  // the captured pass carries the old inverse
    b->inv_method = method;
    cudaSetDevice(b->device);
    return batch_prepare(*b);  // the other inverse's workspace and tables, outside any capture
}

gw_status gw_batch_run(gw_batch *b, int use_graph)
{
    if (!b)
        return GW_E_INVALID;
    gw_batch &bb = *b;
    cudaSetDevice(bb.device);
    for (gw_ctx *h : bb.ctxs)
        if (!h->c.loaded)
            return bfail(bb, GW_E_NOT_READY, "a context lost its states");
    // work queued earlier on the contexts' stream comes first
    GW_BCUDA(cudaStreamSynchronize(bb.ctxs[0]->c.stream), "context stream synchronize");
    if (!use_graph || bb.runs == 0) {
        // eager pass (the first pass is always eager, so every lazy setup happens outside capture)
        const gw_status st = batch_enqueue(bb);
        if (st != GW_OK) {
            cudaStreamSynchronize(bb.stream);
            return st;
        }
    } else {
        if (!bb.exec) {
            cudaStreamCaptureStatus cs;
            if (cudaStreamIsCapturing(bb.stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
                return bfail(bb, GW_E_INVALID, "the batch stream is already being captured");
            if (cudaStreamBeginCapture(bb.stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
                cudaGetLastError();
                return bfail(bb, GW_E_CUDA, "stream capture could not start");
            }
            const unsigned long long counted = g_launches.load();
            const gw_status st = batch_enqueue(bb);
            g_launches.store(counted);  // captured launches run at replay time, where they are counted
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(bb.stream, &g);
            if (st != GW_OK || ec != cudaSuccess || !g) {
                cudaGetLastError();
                if (g)
                    cudaGraphDestroy(g);
                return st != GW_OK ? st : bfail(bb, GW_E_CUDA, "stream capture failed");
            }
            bb.graph = g;
            if (cudaGraphInstantiate(&bb.exec, bb.graph, 0) != cudaSuccess) {
                cudaGetLastError();
                drop_graph(bb);
                return bfail(bb, GW_E_CUDA, "graph instantiation failed");
            }
            bb.graph_kernels = static_cast<int>(kernel_nodes(bb.graph));
        }
        GW_BCUDA(cudaGraphLaunch(bb.exec, bb.stream), "graph launch");
        count_launches(bb.graph_kernels);
    }
    ++bb.runs;
    return batch_status(bb);
}

gw_status gw_batch_autotune(gw_batch *b, const char *cache_path, double target_error)
{
    if (!b || !(target_error > 0.0))
        return GW_E_INVALID;
    gw_batch &bb = *b;
    cudaSetDevice(bb.device);
    // the choice depends on the error target as well as on the shapes, and on the error table
    // of the update kernel (rule2: the three-N=256 + six-N=128 form)
    char tgt[48];
    std::snprintf(tgt, sizeof tgt, "|target%.3g|rule2", target_error);
    const std::string key = batch_key(bb) + tgt;
    if (cache_path) {
        if (FILE *f = std::fopen(cache_path, "r")) {
            char line[8192];
            int W = 0, L = 0;
            while (std::fgets(line, sizeof line, f)) {
                const std::string s(line);
                const std::string want = "{\"key\": \"" + key + "\"";
                if (s.compare(0, want.size(), want) == 0) {
                    const size_t pw = s.find("\"W\": "), pl = s.find("\"L\": ");
                    if (pw != std::string::npos && pl != std::string::npos) {
                        W = std::atoi(s.c_str() + pw + 5);
                        L = std::atoi(s.c_str() + pl + 5);
                    }
                }
            }
            std::fclose(f);
            if (W >= 1 && L >= 1)
                return gw_batch_set_window(b, W, L);
        }
    }
    struct Cand {
        int W, L;
    };
    const Cand cands[] = {{1, 4096}, {2, 256}, {2, 4096}, {3, 4096}, {4, 4096}, {6, 4096}, {8, 4096}};
    GW_TRY(batch_pair_densities(bb));
    int bestW = 0, bestL = 0;
    float best = 1e30f;
    for (const Cand &cd : cands) {
        if (predicted_error(bb.precision, cd.W) * 1.25 > target_error)
            continue;
        bb.W = cd.W;
        bb.L = cd.L;
        GW_TRY(batch_herk(bb));  // warm-up
        float tot = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            GW_TRY(batch_herk(bb));
            GW_BCUDA(cudaEventSynchronize(bb.e1), "autotune sync");
            float ms = 0.f;
            GW_BCUDA(cudaEventElapsedTime(&ms, bb.e0, bb.e1), "autotune timing");
            tot += ms;
        }
        if (tot < best) {
            best = tot;
            bestW = cd.W;
            bestL = cd.L;
        }
    }
    const gw_status st = batch_status(bb);
    if (st != GW_OK)
        return st;
    if (bestW == 0)
        return bfail(bb, GW_E_UNSUPPORTED, "no window length meets error target %g", target_error);
    drop_graph(bb);
    bb.W = bestW;
    bb.L = bestL;
    if (cache_path) {
        if (FILE *f = std::fopen(cache_path, "a")) {
            std::fprintf(f, "{\"key\": \"%s\", \"W\": %d, \"L\": %d, \"herk_ms\": %.4f, \"target_error\": %g}\n",
                         key.c_str(), bestW, bestL, best / 2.f, target_error);
            std::fclose(f);
        }
    }
    return GW_OK;
}

gw_status gw_batch_stats(gw_batch *b, double *stats4)
{
    if (!b || !stats4)
        return GW_E_INVALID;
    stats4[0] = b->herk_ms;
    stats4[1] = b->W;
    stats4[2] = b->L;
    stats4[3] = b->n_tiles;
    return GW_OK;
}

gw_status gw_batch_last_error(const gw_batch *b, char *buf, size_t n)
{
    if (!b || !buf || n == 0)
        return GW_E_INVALID;
    std::snprintf(buf, n, "%s", b->last_error.c_str());
    return GW_OK;
}

}  // extern "C"
