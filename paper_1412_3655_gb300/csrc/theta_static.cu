// culgt_theta_static_scratch: theta and F of a canonical link buffer without
// any device allocation.
//
// Some callers cannot allocate device memory while they run: a host program
// that has handed the whole GPU to its own memory pool (so cudaMalloc fails or
// fragments that pool), or a stream-ordered loop that cannot afford the
// device-wide synchronisation cudaMalloc/cudaFree may cause. For them this
// entry point reads the caller's canonical links directly (no internal
// layout copy) and keeps its per-block partial sums in a fixed, file-scope
// device array instead of handle scratch. The caller passes the links and a
// device buffer for the two results.
//
// The array holds kMaxPartials partial sums (256 KB), one per block of 256
// sites, so lattices up to kMaxSites = 4,194,304 sites are accepted. Every
// GPU that loads this library holds the array until the process exits. All
// calls share it: each call overwrites the partials it reads, so nothing
// needs clearing, but calls that overlap on the GPU (different streams or
// host threads) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/culgt.h"
#include "kernels.cuh"
#include "launch.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxPartials = 16384;
constexpr long long kMaxSites = (long long)kMaxPartials * kThreads;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double2 g_theta_scratch[kMaxPartials];

// Device address of g_theta_scratch on each device, looked up with that
// device current. Host code may not pass the symbol itself to a kernel: on the
// host it names a stand-in, not device memory. The address belongs to the
// device's current CUDA context; cudaDeviceReset destroys that context and the
// next one may load the array elsewhere, so the address is cached together
// with the context's unique id (cuCtxGetId, reached through the runtime's
// driver entry points, no link to libcuda) and looked up again when the id
// changes.
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);

std::mutex g_setup_mutex;
double2 *g_scratch_addr[kMaxDevices];
unsigned long long g_scratch_ctx[kMaxDevices];
CtxGetCurrentFn g_ctx_get_current;
CtxGetIdFn g_ctx_get_id;

// id of the calling thread's current context, 0 if none (or not available)
unsigned long long current_context_id()
{
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
            (void)cudaGetLastError();
            return 0;
        }
        g_ctx_get_current = (CtxGetCurrentFn)f1;
        g_ctx_get_id = (CtxGetIdFn)f2;
    }
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != 0 || !ctx || g_ctx_get_id(ctx, &id) != 0) return 0;
    return id;
}

culgt_status scratch_for_current_device(double2 **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        return CULGT_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long id = current_context_id();
    if (!g_scratch_addr[dev] || id == 0 || id != g_scratch_ctx[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_theta_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return CULGT_ERR_CUDA;
        }
        g_scratch_addr[dev] = (double2 *)p;
        // the lookup makes the device's primary context current if none was
        g_scratch_ctx[dev] = current_context_id();
    }
    *out = g_scratch_addr[dev];
    return CULGT_OK;
}

// tr[Delta Delta^+] of one site from the canonical links, in FP64, for any
// Nc: Delta = [(M - M^+)/(2i)]_traceless with M = sum_mu U_mu(x) - U_mu(x-mu)
template <typename In, int NC>
__global__ void __launch_bounds__(kThreads) k_theta_canonical(const In *canon, culgt::Geom g, double2 *partials)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double th = 0.0, fs = 0.0;
    if (i < g.V) {
        int x[4];
        x[1] = i % g.L[1];
        int r = i / g.L[1];
        x[2] = r % g.L[2];
        r /= g.L[2];
        x[3] = r % g.L[3];
        x[0] = r / g.L[3];
        double mr[NC][NC], mi[NC][NC];
#pragma unroll
        for (int a = 0; a < NC; a++)
#pragma unroll
            for (int b = 0; b < NC; b++) mr[a][b] = mi[a][b] = 0.0;
        const int stride[4] = {g.L[1] * g.L[2] * g.L[3], 1, g.L[1], g.L[1] * g.L[2]};
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            int ib = x[mu] == 0 ? i + (g.L[mu] - 1) * stride[mu] : i - stride[mu];
            const In *f = canon + ((size_t)i * 4 + mu) * (2 * NC * NC);
            const In *bk = canon + ((size_t)ib * 4 + mu) * (2 * NC * NC);
#pragma unroll
            for (int a = 0; a < NC; a++) {
                fs += (double)f[2 * (a * NC + a)];
#pragma unroll
                for (int b = 0; b < NC; b++) {
                    mr[a][b] += (double)f[2 * (a * NC + b)] - (double)bk[2 * (a * NC + b)];
                    mi[a][b] += (double)f[2 * (a * NC + b) + 1] - (double)bk[2 * (a * NC + b) + 1];
                }
            }
        }
        double tr = 0.0;
#pragma unroll
        for (int a = 0; a < NC; a++) tr += mi[a][a];
#pragma unroll
        for (int a = 0; a < NC; a++) {
            double d = mi[a][a] - tr / NC;
            th += d * d;
#pragma unroll
            for (int b = a + 1; b < NC; b++) {
                double zr = mr[a][b] - mr[b][a], zi = mi[a][b] + mi[b][a];
                th += 0.5 * (zr * zr + zi * zi);
            }
        }
    }
    culgt::block_reduce2(th, fs, partials);
}

} // namespace

extern "C" culgt_status culgt_theta_static_scratch(const void *d_links, const culgt_params *p, void *cuda_stream,
                                                   double *d_out)
{
    culgt_status st = culgt_validate(p);
    if (st != CULGT_OK) return st;
    if (p->gauge != CULGT_LANDAU) return CULGT_ERR_ARG;
    if (!d_links || !d_out) return CULGT_ERR_ARG;
    long long V = (long long)p->dims[0] * p->dims[1] * p->dims[2] * p->dims[3];
    if (V > kMaxSites) return CULGT_ERR_TOO_LARGE;
    double2 *scratch = nullptr;
    st = scratch_for_current_device(&scratch);
    if (st != CULGT_OK) return st;
    culgt::Geom g;
    for (int mu = 0; mu < 4; mu++) g.L[mu] = p->dims[mu];
    g.half1 = g.L[1] / 2;
    g.V = (int)V;
    g.Vh = (int)(V / 2);
    g.stride = 0;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int nb = (int)((V + kThreads - 1) / kThreads);
    if (p->nc == 3 && p->dtype_in == 0)
        k_theta_canonical<double, 3><<<nb, kThreads, 0, s>>>((const double *)d_links, g, scratch);
    else if (p->nc == 3)
        k_theta_canonical<float, 3><<<nb, kThreads, 0, s>>>((const float *)d_links, g, scratch);
    else if (p->dtype_in == 0)
        k_theta_canonical<double, 2><<<nb, kThreads, 0, s>>>((const double *)d_links, g, scratch);
    else
        k_theta_canonical<float, 2><<<nb, kThreads, 0, s>>>((const float *)d_links, g, scratch);
    culgt::count_launch();
    culgt::launch_finalize2(scratch, nb, 1.0 / (double)V, 1.0 / (4.0 * p->nc * (double)V), d_out, s);
    if (cudaGetLastError() != cudaSuccess) return CULGT_ERR_CUDA;
    return CULGT_OK;
}
