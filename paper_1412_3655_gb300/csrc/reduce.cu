// Deterministic final stage of the FP64 reductions and the Ops lookup.
#include <atomic>

#include "kernels.cuh"
#include "launch.h"

namespace culgt {

static std::atomic<long long> g_launches{0};

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

// one block of 256 threads: thread t sums partials t, t+256, ... in order,
// then a fixed shuffle tree; the result depends only on n and the partials
__global__ void __launch_bounds__(256) k_finalize2(const double2 *partials, int n, double sx, double sy, double *out)
{
    __shared__ double sa[8], sb[8];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        a += partials[k].x;
        b += partials[k].y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int k = 0; k < 8; k++) {
            ta += sa[k];
            tb += sb[k];
        }
        out[0] = ta * sx;
        out[1] = tb * sy;
    }
}

__global__ void __launch_bounds__(256) k_finalize_max(const double2 *partials, int n, double *out)
{
    __shared__ double sm[8];
    double m = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) m = fmax(m, partials[k].x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < 8; k++) t = fmax(t, sm[k]);
        out[0] = t;
    }
}

void launch_finalize_max(const double2 *partials, int n, double *out, cudaStream_t s)
{
    k_finalize_max<<<1, 256, 0, s>>>(partials, n, out);
    count_launch();
}

void launch_finalize2(const double2 *partials, int n, double sx, double sy, double *out, cudaStream_t s)
{
    k_finalize2<<<1, 256, 0, s>>>(partials, n, sx, sy, out);
    count_launch();
}

int max_partials(const Geom &g)
{
    // theta (256 threads) and plaquette (128 threads) over 2 Vh sites,
    // unitarity (256 threads) over 8 Vh links
    long long a = (2LL * g.Vh + 127) / 128, b = (8LL * g.Vh + 255) / 256;
    return (int)(a > b ? a : b);
}

const Ops *get_ops_df(int nc) { return nc == 3 ? &ops_su3_df18 : &ops_su2_df4; }

const Ops *get_ops(int nc, int fp32, int nreal)
{
    if (nc == 3 && !fp32 && nreal == 18) return &ops_su3_d18;
    if (nc == 3 && !fp32 && nreal == 12) return &ops_su3_d12;
    if (nc == 3 && fp32 && nreal == 12) return &ops_su3_f12;
    if (nc == 3 && fp32 && nreal == 18) return &ops_su3_f18;
    if (nc == 2 && !fp32 && nreal == 4) return &ops_su2_d4;
    if (nc == 2 && fp32 && nreal == 4) return &ops_su2_f4;
    return nullptr;
}

} // namespace culgt
