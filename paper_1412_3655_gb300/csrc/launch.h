// Host-side launch interface between the C ABI (api.cu) and the kernel
// instantiations (ops_*.cu). One Ops table per storage parameterisation.
#pragma once

#include <cuda_runtime.h>

#include "culgt_device.cuh"

namespace culgt {

// switch_theta = 0 (automatic switch of the mixed schedules): the FP32 phase
// goes past this theta for as long as every check interval still lowers
// theta, and switches at the first that does not (the FP32 rounding floor)
constexpr double kAutoSwitchFloor = 1e-8;

// geometry of an L0 x L1 x L2 x L3 lattice in the internal layout
inline Geom make_geom(const int *dims)
{
    Geom g;
    for (int mu = 0; mu < 4; mu++) g.L[mu] = dims[mu];
    g.half1 = dims[1] / 2;
    g.V = dims[0] * dims[1] * dims[2] * dims[3];
    g.Vh = g.V / 2;
    g.stride = ((size_t)g.Vh + 63) / 64 * 64;
    return g;
}

struct Ops {
    int nc;         // 2 or 3
    int nreal;      // reals per link in device memory
    int fp32;       // 1 if the links are float
    int df;         // 1 if the links are double-float pairs
    int nchunk;     // chunks per link
    int chunk_bytes;
    // one checkerboard half-sweep of the given parity, tps (1 or 2) threads per
    // site in blocks of `block` threads, minb blocks of 128 per SM (1: no
    // register cap; 3 or 4: block must be 128); gacc != null (FP32 storage)
    // also accumulates g(x) per site. Every mapping gives the same result.
    void (*halfsweep)(void *base, void *gacc, const Geom &g, int parity, double omega, int variant, int tps,
                      int block, int minb, cudaStream_t s);
    // one heat-bath half-sweep of the given parity at temperature 1/inv_temp
    // (simulated annealing), draws keyed by (k0, k1) with sweep word `sweep`;
    // one thread per site, blocks of 128; gacc as in halfsweep. variant picks
    // one of heatbath_variants mappings (registers held / capped), all giving
    // the same links.
    void (*heatbath)(void *base, void *gacc, const Geom &g, int parity, double inv_temp, uint32_t k0, uint32_t k1,
                     uint32_t sweep, int variant, cudaStream_t s);
    int heatbath_variants;
    void (*heatbath_mapping)(int variant, int *keep_links, int *min_blocks_per_sm);
    // one maximally Abelian gauge half-sweep (1 thread per site, blocks of
    // 128); gacc as in halfsweep
    void (*mag_halfsweep)(void *base, void *gacc, const Geom &g, int parity, double omega, int variant,
                          cudaStream_t s);
    // one MAG heat-bath half-sweep (simulated annealing), as heatbath
    void (*mag_heatbath)(void *base, void *gacc, const Geom &g, int parity, double inv_temp, uint32_t k0, uint32_t k1,
                         uint32_t sweep, cudaStream_t s);
    // per-block partial sums of (theta_MAG site terms, sum_mu sum_a |U_aa|^2); returns the block count
    int (*mag_theta_partials)(const void *base, const Geom &g, double2 *partials, cudaStream_t s);
    // per-block partial sums of (tr Delta Delta^+, sum Re tr U) over all sites; returns the block count
    int (*theta_partials)(const void *base, const Geom &g, int mu_first, double2 *partials, cudaStream_t s);
    // per-block partial sums of the plaquette trace; returns the block count
    int (*plaq_partials)(const void *base, const Geom &g, double2 *partials, cudaStream_t s);
    void (*reunitarize)(void *base, const Geom &g, cudaStream_t s);
    void (*gauge_identity)(void *gacc, const Geom &g, cudaStream_t s);
    void (*gauge_reunitarize)(void *gacc, const Geom &g, cudaStream_t s);
    int gauge_nchunk;     // chunks per site of the FP32 accumulator (0 for FP64 storage)
    int gauge_chunk_bytes;
    // per-block max of |U U^+ - 1| over all links; returns the block count
    int (*unitarity_partials)(const void *base, const Geom &g, double2 *partials, cudaStream_t s);
    void (*to_internal_d)(const double *canon, void *base, const Geom &g, cudaStream_t s);
    void (*to_internal_f)(const float *canon, void *base, const Geom &g, cudaStream_t s);
    void (*to_canonical_d)(const void *base, double *canon, const Geom &g, cudaStream_t s);
    void (*to_canonical_f)(const void *base, float *canon, const Geom &g, cudaStream_t s);
};

// host-side count of kernel launches (culgt_kernel_launches)
void count_launch(int n = 1);
long long launches_so_far();

// nullptr if the combination is not built
const Ops *get_ops(int nc, int fp32, int nreal);

// FP64 links <- g(x) U g(x+mu)^+ with g from the FP32 accumulator of `from`
void launch_rotate_orbit(const Ops *from, const void *gacc, const Ops *to, void *base64, const Geom &g,
                         cudaStream_t s);

// largest number of partials any reduction launch writes for this geometry
int max_partials(const Geom &g);

// out[0] = max_k partials[k].x
void launch_finalize_max(const double2 *partials, int n, double *out, cudaStream_t s);

// out[0] = sx * sum_k partials[k].x, out[1] = sy * sum_k partials[k].y, fixed order
void launch_finalize2(const double2 *partials, int n, double sx, double sy, double *out, cudaStream_t s);

extern const Ops ops_su3_d18, ops_su3_d12, ops_su3_f12, ops_su3_f18, ops_su2_d4, ops_su2_f4, ops_su3_df18,
    ops_su2_df4;

// double-float storage (18 reals for SU(3), quaternion for SU(2))
const Ops *get_ops_df(int nc);

} // namespace culgt
