// The C ABI of libculgt (include/culgt.h): argument checks, the handle, and
// the host drivers of the iteration of Sec. 2 (half-sweeps, theta checks,
// reunitarisation, the FP32 -> FP64 schedule).
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>

#include "../../include/culgt.h"
#include "launch.h"

using namespace culgt;

// CUDA graphs of a handle's check intervals, keyed by (phase, k,
// reunitarisation offsets): graph exec and the number of kernels in it
struct GraphCache {
    std::map<long long, std::pair<cudaGraphExec_t, int>> exec;
    ~GraphCache()
    {
        for (auto &kv : exec) cudaGraphExecDestroy(kv.second.first);
    }
};

struct culgt_handle {
    culgt_params prm;
    cudaStream_t stream;   // the handle's own stream: all of its work, and graph capture
    cudaStream_t ustream;  // the caller's stream, ordered against `stream` by events at every call
    cudaEvent_t ev_in, ev_out;
    GraphCache *graphs;
    Geom geom;
    const Ops *ops32;  // FP32 storage (FP32 and mixed), else null
    const Ops *ops64;  // FP64 storage (FP64 and mixed), else null
    void *buf32;
    void *buf64;
    int cur32;         // 1 while the FP32 buffer holds the current links
    int loaded;
    double2 *partials;
    double *d_scalars;  // 4 doubles
    double *h_scalars;  // pinned, 4 doubles
    void *staging;      // canonical device buffer for the host entry point
    void *gacc;         // mixed: FP32 accumulated gauge transformation per site
    int sweeps32, sweeps64;
    // half-sweep mapping per precision: threads per site, block, blocks per SM (0 = not chosen yet)
    int tps32, block32, minb32, tps64, block64, minb64;
    // heat-bath mapping per precision (variant + 1; 0 = not chosen yet)
    int hb32, hb64;
};

namespace {

#define CU(call)                                        \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) {                        \
            (void)cudaGetLastError();                   \
            return CULGT_ERR_CUDA;                      \
        }                                               \
    } while (0)

#define ST(call)                                        \
    do {                                                \
        culgt_status s_ = (call);                       \
        if (s_ < 0) return s_;                          \
    } while (0)

int default_storage(int nc, int fp32) { return nc == 2 ? 4 : (fp32 ? 12 : 18); }

// Work of a handle call runs on the handle's own stream, after everything
// already queued on the caller's stream, and the caller's stream waits for it.
struct CallScope {
    culgt_handle *h;
    explicit CallScope(culgt_handle *hh) : h(hh)
    {
        cudaEventRecord(h->ev_in, h->ustream);
        cudaStreamWaitEvent(h->stream, h->ev_in, 0);
    }
    ~CallScope()
    {
        cudaEventRecord(h->ev_out, h->stream);
        cudaStreamWaitEvent(h->ustream, h->ev_out, 0);
    }
};

culgt_status validate(const culgt_params *p)
{
    if (!p) return CULGT_ERR_ARG;
    if (p->nc != 2 && p->nc != 3) return CULGT_ERR_NC;
    long long V = 1;
    for (int mu = 0; mu < 4; mu++) {
        if (p->dims[mu] < 2 || (p->dims[mu] & 1)) return CULGT_ERR_DIMS;
        V *= p->dims[mu];
    }
    if (V >= (1LL << 31) / 4) return CULGT_ERR_DIMS;
    if (!(p->omega >= 1.0 && p->omega < 2.0)) return CULGT_ERR_ARG;
    if (p->or_variant != 0 && p->or_variant != 1) return CULGT_ERR_ARG;
    if (p->precision < CULGT_FP64 || p->precision > CULGT_DF) return CULGT_ERR_ARG;
    if (p->nc == 3 && p->storage_reals != 0 && p->storage_reals != 12 && p->storage_reals != 18) return CULGT_ERR_NC;
    if (p->nc == 2 && p->storage_reals != 0 && p->storage_reals != 4) return CULGT_ERR_NC;
    if (!(p->theta_target >= 0.0) || std::isinf(p->theta_target)) return CULGT_ERR_ARG;
    if (p->max_sweeps < 0 || p->check_every < 1 || p->reunit_every < 0) return CULGT_ERR_ARG;
    if ((p->precision == CULGT_MIXED || p->precision == CULGT_MIXED_DF) &&
        !(p->switch_theta > 0.0 || p->switch_theta == 0.0))
        return CULGT_ERR_ARG;
    if (p->dtype_in != 0 && p->dtype_in != 1) return CULGT_ERR_ARG;
    if (p->threads_per_site < 0 || p->threads_per_site > 2) return CULGT_ERR_ARG;
    if (p->block_size != 0 && p->block_size != 64 && p->block_size != 128 && p->block_size != 256) return CULGT_ERR_ARG;
    if (p->min_blocks_per_sm != 0 && p->min_blocks_per_sm != 1 && p->min_blocks_per_sm != 3 &&
        p->min_blocks_per_sm != 4)
        return CULGT_ERR_ARG;
    if (p->gauge != CULGT_LANDAU && p->gauge != CULGT_MAG) return CULGT_ERR_ARG;
    return CULGT_OK;
}

// the Landau-only entry points (one-call Landau, Coulomb, batched, annealing)
culgt_status validate_landau(const culgt_params *p)
{
    culgt_status st = validate(p);
    if (st != CULGT_OK) return st;
    return p->gauge == CULGT_LANDAU ? CULGT_OK : CULGT_ERR_ARG;
}

size_t buffer_bytes(const Ops *o, const Geom &g) { return (size_t)8 * o->nchunk * g.stride * o->chunk_bytes; }

void pick_ops(const culgt_params *p, const Ops **o32, const Ops **o64)
{
    *o32 = *o64 = nullptr;
    const int sr32 = p->storage_reals ? p->storage_reals : default_storage(p->nc, 1);
    switch (p->precision) {
    case CULGT_FP64: *o64 = get_ops(p->nc, 0, p->storage_reals ? p->storage_reals : default_storage(p->nc, 0)); break;
    case CULGT_FP32: *o32 = get_ops(p->nc, 1, sr32); break;
    case CULGT_MIXED:
        *o32 = get_ops(p->nc, 1, sr32);
        *o64 = get_ops(p->nc, 0, default_storage(p->nc, 0));
        break;
    case CULGT_MIXED_DF:
        *o32 = get_ops(p->nc, 1, sr32);
        *o64 = get_ops_df(p->nc);
        break;
    default: *o64 = get_ops_df(p->nc); break;
    }
}

size_t gauge_bytes(const Ops *o32, const Geom &g)
{
    return (size_t)2 * o32->gauge_nchunk * g.stride * o32->gauge_chunk_bytes;
}

size_t canonical_bytes(const culgt_params *p, const Geom &g)
{
    return (size_t)g.V * 4 * p->nc * p->nc * 2 * (p->dtype_in ? sizeof(float) : sizeof(double));
}

const Ops *cur_ops(const culgt_handle *h) { return h->cur32 ? h->ops32 : h->ops64; }
void *cur_buf(const culgt_handle *h) { return h->cur32 ? h->buf32 : h->buf64; }

culgt_status sync_scalars(culgt_handle *h, int n)
{
    CU(cudaMemcpyAsync(h->h_scalars, h->d_scalars, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    CU(cudaGetLastError());
    return CULGT_OK;
}

// queue theta and F of the current links into h_scalars (pinned host)
void theta_enqueue(culgt_handle *h)
{
    const Geom &g = h->geom;
    int nb = h->prm.gauge == CULGT_MAG ? cur_ops(h)->mag_theta_partials(cur_buf(h), g, h->partials, h->stream)
                                       : cur_ops(h)->theta_partials(cur_buf(h), g, 0, h->partials, h->stream);
    launch_finalize2(h->partials, nb, 1.0 / g.V, 1.0 / (4.0 * h->prm.nc * g.V), h->d_scalars, h->stream);
    cudaMemcpyAsync(h->h_scalars, h->d_scalars, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
}

// theta and F of the current links, normalised as in the header (Landau)
culgt_status theta_now(culgt_handle *h, double *theta, double *F)
{
    theta_enqueue(h);
    CU(cudaStreamSynchronize(h->stream));
    CU(cudaGetLastError());
    *theta = h->h_scalars[0];
    *F = h->h_scalars[1];
    if (!std::isfinite(*theta) || !std::isfinite(*F)) return CULGT_ERR_NONFINITE;
    return CULGT_OK;
}

// of the current links, or with fp64 = true of the FP64 buffer (a mixed
// handle's FP64 input before the switch)
culgt_status plaquette_now(culgt_handle *h, double *P, bool fp64 = false)
{
    const Geom &g = h->geom;
    const Ops *o = fp64 ? h->ops64 : cur_ops(h);
    const void *b = fp64 ? h->buf64 : cur_buf(h);
    int nb = o->plaq_partials(b, g, h->partials, h->stream);
    launch_finalize2(h->partials, nb, 1.0 / (6.0 * h->prm.nc * g.V), 0.0, h->d_scalars, h->stream);
    ST(sync_scalars(h, 1));
    *P = h->h_scalars[0];
    return CULGT_OK;
}

culgt_status unitarity_now(culgt_handle *h, double *err)
{
    int nb = cur_ops(h)->unitarity_partials(cur_buf(h), h->geom, h->partials, h->stream);
    launch_finalize_max(h->partials, nb, h->d_scalars, h->stream);
    ST(sync_scalars(h, 1));
    *err = h->h_scalars[0];
    return CULGT_OK;
}

// Autotuner (the paper's runtime choice of kernel settings, Sec. 5): each
// (threads per site, block size) mapping is timed on a scratch copy of the
// links; the first one in list order within 2% of the fastest is kept per
// (storage, lattice volume, accumulation) for the process. All mappings give
// bitwise identical links, so the choice never changes a result. Lattices
// below kTuneMinSites use the default mapping.
constexpr int kTuneMinSites = 1 << 16;
constexpr float kTuneSlack = 1.02f;
std::mutex g_tune_mutex;

struct Mapping {
    int tps, block, minb;
};
std::map<std::tuple<const Ops *, int, bool, int>, Mapping> g_tune_cache;

// the mappings the autotuner tries (the paper's axes: threads per site and a
// register limit through __launch_bounds__; plus the block size)
const Mapping kMappings[] = {{1, 64, 1}, {1, 128, 1}, {1, 256, 1}, {1, 128, 3}, {1, 128, 4},
                             {2, 64, 1},  {2, 128, 1}, {2, 256, 1}, {2, 128, 4}};

bool mapping_allowed(const culgt_params &p, const Mapping &m)
{
    if (p.threads_per_site && m.tps != p.threads_per_site) return false;
    if (p.block_size && m.block != p.block_size) return false;
    if (p.min_blocks_per_sm && m.minb != p.min_blocks_per_sm) return false;
    return true;
}

// scratch copy and timing events of a tuner, released on every return path
struct TuneScratch {
    void *p = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    culgt_status init(size_t bytes)
    {
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            p = nullptr;
            return CULGT_ERR_OOM;
        }
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            (void)cudaGetLastError();
            return CULGT_ERR_CUDA;
        }
        return CULGT_OK;
    }
    ~TuneScratch()
    {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (p) cudaFree(p);
    }
};

culgt_status autotune(culgt_handle *h, const Ops *o, void *buf, bool acc, Mapping *out)
{
    const culgt_params &p = h->prm;
    int n_allowed = 0;
    Mapping only = {1, 128, 1};
    for (const Mapping &m : kMappings)
        if (mapping_allowed(p, m)) {
            if (!n_allowed) only = m;
            n_allowed++;
        }
    if (!n_allowed) return CULGT_ERR_ARG;
    if (n_allowed == 1 || h->geom.V < kTuneMinSites) {
        // small lattices: the first allowed mapping in the list
        *out = only;
        return CULGT_OK;
    }
    auto key = std::make_tuple(o, h->geom.V, acc, p.threads_per_site * 10000 + p.block_size * 10 + p.min_blocks_per_sm);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *out = it->second;
            return CULGT_OK;
        }
    }
    size_t bytes = buffer_bytes(o, h->geom);
    size_t gbytes = acc ? gauge_bytes(o, h->geom) : 0;
    TuneScratch ts;
    ST(ts.init(bytes + gbytes));
    void *scratch = ts.p, *gscratch = acc ? (char *)ts.p + bytes : nullptr;
    cudaEvent_t e0 = ts.e0, e1 = ts.e1;
    CU(cudaMemcpyAsync(scratch, buf, bytes, cudaMemcpyDeviceToDevice, h->stream));
    if (acc) CU(cudaMemcpyAsync(gscratch, h->gacc, gbytes, cudaMemcpyDeviceToDevice, h->stream));
    float times[sizeof(kMappings) / sizeof(kMappings[0])];
    float best = 1e30f;
    int idx = 0;
    for (const Mapping &m : kMappings) {
        times[idx] = 1e30f;
        if (mapping_allowed(p, m)) {
            o->halfsweep(scratch, gscratch, h->geom, 0, p.omega, p.or_variant, m.tps, m.block, m.minb, h->stream);
            cudaEventRecord(e0, h->stream);
            for (int r = 0; r < 2; r++)
                for (int parity = 0; parity < 2; parity++)
                    o->halfsweep(scratch, gscratch, h->geom, parity, p.omega, p.or_variant, m.tps, m.block, m.minb,
                                 h->stream);
            cudaEventRecord(e1, h->stream);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&times[idx], e0, e1);
            count_launch(-5);  // tuning launches are not part of the caller's work
            if (times[idx] < best) best = times[idx];
        }
        idx++;
    }
    // the first mapping (list order) within kTuneSlack of the fastest: timing
    // noise between near-equal mappings does not flip the choice
    Mapping pick = only;
    for (int k = 0; k < idx; k++)
        if (times[k] <= best * kTuneSlack) {
            pick = kMappings[k];
            break;
        }
    CU(cudaGetLastError());
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = pick;
    }
    *out = pick;
    return CULGT_OK;
}

culgt_status tuned_mapping(culgt_handle *h, Mapping *m)
{
    const bool acc = h->cur32 && h->gacc;
    int *t = h->cur32 ? &h->tps32 : &h->tps64;
    int *b = h->cur32 ? &h->block32 : &h->block64;
    int *n = h->cur32 ? &h->minb32 : &h->minb64;
    if (!*t) {
        Mapping pick;
        ST(autotune(h, cur_ops(h), cur_buf(h), acc, &pick));
        *t = pick.tps;
        *b = pick.block;
        *n = pick.minb;
    }
    *m = {*t, *b, *n};
    return CULGT_OK;
}

// In the FP32 phase of a mixed handle the half-sweeps also accumulate g(x).
culgt_status sweep_now(culgt_handle *h, int n)
{
    const Ops *o = cur_ops(h);
    void *b = cur_buf(h);
    void *acc = (h->cur32 && h->gacc) ? h->gacc : nullptr;
    if (h->prm.gauge == CULGT_MAG) {
        for (int k = 0; k < n; k++)
            for (int parity = 0; parity < 2; parity++)
                o->mag_halfsweep(b, acc, h->geom, parity, h->prm.omega, h->prm.or_variant, h->stream);
        return CULGT_OK;
    }
    Mapping m;
    ST(tuned_mapping(h, &m));
    for (int k = 0; k < n; k++)
        for (int parity = 0; parity < 2; parity++)
            o->halfsweep(b, acc, h->geom, parity, h->prm.omega, h->prm.or_variant, m.tps, m.block, m.minb, h->stream);
    return CULGT_OK;
}

void reunitarize_now(culgt_handle *h)
{
    cur_ops(h)->reunitarize(cur_buf(h), h->geom, h->stream);
    if (h->cur32 && h->gacc) h->ops32->gauge_reunitarize(h->gacc, h->geom, h->stream);
}

// ---- simulated annealing: heat-bath and microcanonical sweeps ----

culgt_status validate_anneal(const culgt_anneal_params *a)
{
    if (!a) return CULGT_ERR_ARG;
    if (!(a->t_start > 0.0) || !(a->t_end > 0.0) || std::isinf(a->t_start) || std::isinf(a->t_end))
        return CULGT_ERR_ARG;
    if (a->steps < 0 || a->micro_sweeps < 0) return CULGT_ERR_ARG;
    return CULGT_OK;
}

// T_k of the schedule, linear in k from t_start to t_end
double anneal_temperature(const culgt_anneal_params *a, int k)
{
    return a->steps > 1 ? a->t_start + (a->t_end - a->t_start) * (double)k / (double)(a->steps - 1) : a->t_start;
}

// The heat-bath mapping, timed like the half-sweep's (autotune): every
// variant on a scratch copy, the fastest kept per (storage, volume,
// accumulation) for the process; lattices below kTuneMinSites take variant 0.
std::map<std::tuple<const Ops *, int, bool>, int> g_hb_cache;

culgt_status tuned_heatbath(culgt_handle *h, int *variant)
{
    int *slot = h->cur32 ? &h->hb32 : &h->hb64;
    if (*slot) {
        *variant = *slot - 1;
        return CULGT_OK;
    }
    const Ops *o = cur_ops(h);
    const bool acc = h->cur32 && h->gacc;
    int pick = 0;
    if (o->heatbath_variants > 1 && h->geom.V >= kTuneMinSites) {
        auto key = std::make_tuple(o, h->geom.V, acc);
        bool cached = false;
        {
            std::lock_guard<std::mutex> lock(g_tune_mutex);
            auto it = g_hb_cache.find(key);
            if (it != g_hb_cache.end()) {
                pick = it->second;
                cached = true;
            }
        }
        if (!cached) {
            size_t bytes = buffer_bytes(o, h->geom);
            size_t gbytes = acc ? gauge_bytes(o, h->geom) : 0;
            TuneScratch ts;
            ST(ts.init(bytes + gbytes));
            void *scratch = ts.p, *gscratch = acc ? (char *)ts.p + bytes : nullptr;
            cudaEvent_t e0 = ts.e0, e1 = ts.e1;
            CU(cudaMemcpyAsync(scratch, cur_buf(h), bytes, cudaMemcpyDeviceToDevice, h->stream));
            if (acc) CU(cudaMemcpyAsync(gscratch, h->gacc, gbytes, cudaMemcpyDeviceToDevice, h->stream));
            float best = 1e30f, times[8];
            const int nv = o->heatbath_variants < 8 ? o->heatbath_variants : 8;
            for (int v = 0; v < nv; v++) {
                o->heatbath(scratch, gscratch, h->geom, 0, 1.0, 0u, 0u, 0u, v, h->stream);
                cudaEventRecord(e0, h->stream);
                for (int r = 0; r < 2; r++)
                    for (int parity = 0; parity < 2; parity++)
                        o->heatbath(scratch, gscratch, h->geom, parity, 1.0, 0u, 0u, (unsigned)r, v, h->stream);
                cudaEventRecord(e1, h->stream);
                cudaEventSynchronize(e1);
                times[v] = 0.0f;
                cudaEventElapsedTime(&times[v], e0, e1);
                count_launch(-5);  // tuning launches are not part of the caller's work
                if (times[v] < best) best = times[v];
            }
            for (int v = 0; v < nv; v++)
                if (times[v] <= best * kTuneSlack) {
                    pick = v;
                    break;
                }
            CU(cudaGetLastError());
            std::lock_guard<std::mutex> lock(g_tune_mutex);
            g_hb_cache[key] = pick;
        }
    }
    *slot = pick + 1;
    *variant = pick;
    return CULGT_OK;
}

culgt_status heatbath_now(culgt_handle *h, double T, unsigned long long seed, unsigned sweep)
{
    const Ops *o = cur_ops(h);
    void *acc = (h->cur32 && h->gacc) ? h->gacc : nullptr;
    if (h->prm.gauge == CULGT_MAG) {
        for (int parity = 0; parity < 2; parity++)
            o->mag_heatbath(cur_buf(h), acc, h->geom, parity, 1.0 / T, (uint32_t)seed, (uint32_t)(seed >> 32), sweep,
                            h->stream);
        return CULGT_OK;
    }
    int v;
    ST(tuned_heatbath(h, &v));
    for (int parity = 0; parity < 2; parity++)
        o->heatbath(cur_buf(h), acc, h->geom, parity, 1.0 / T, (uint32_t)seed, (uint32_t)(seed >> 32), sweep, v,
                    h->stream);
    return CULGT_OK;
}

// overrelaxation at omega = 2 (r -> r^2 per subgroup keeps Re tr[r w]; for
// MAG the smallest rotation applied twice keeps the block functional)
culgt_status micro_now(culgt_handle *h)
{
    if (h->prm.gauge == CULGT_MAG) {
        void *acc = (h->cur32 && h->gacc) ? h->gacc : nullptr;
        for (int parity = 0; parity < 2; parity++)
            cur_ops(h)->mag_halfsweep(cur_buf(h), acc, h->geom, parity, 2.0, 0, h->stream);
        return CULGT_OK;
    }
    Mapping m;
    ST(tuned_mapping(h, &m));
    const Ops *o = cur_ops(h);
    void *acc = (h->cur32 && h->gacc) ? h->gacc : nullptr;
    for (int parity = 0; parity < 2; parity++)
        o->halfsweep(cur_buf(h), acc, h->geom, parity, 2.0, 0, m.tps, m.block, m.minb, h->stream);
    return CULGT_OK;
}

culgt_status anneal_now(culgt_handle *h, const culgt_anneal_params *a)
{
    long long done = 0;
    for (int k = 0; k < a->steps; k++) {
        const double T = anneal_temperature(a, k);
        for (int m = 0; m <= a->micro_sweeps; m++) {
            if (m == 0)
                ST(heatbath_now(h, T, a->seed, (unsigned)k));
            else
                ST(micro_now(h));
            done++;
            if (h->prm.reunit_every > 0 && done % h->prm.reunit_every == 0) reunitarize_now(h);
        }
    }
    CU(cudaGetLastError());
    return CULGT_OK;
}

// One check interval: k sweeps (reunitarising after sweep n + j when due)
// and the theta of the result, queued into h_scalars.
culgt_status interval_enqueue(culgt_handle *h, int k, int n)
{
    for (int j = 0; j < k; j++) {
        ST(sweep_now(h, 1));
        if (h->prm.reunit_every > 0 && (n + j + 1) % h->prm.reunit_every == 0) reunitarize_now(h);
    }
    theta_enqueue(h);
    return CULGT_OK;
}

// replay the interval's graph, capturing it on first use (after the
// autotuner has fixed the mapping, which the capture must not time)
culgt_status run_interval(culgt_handle *h, int k, int n)
{
    Mapping m;
    if (h->prm.gauge == CULGT_LANDAU) ST(tuned_mapping(h, &m));
    long long mask = 0;
    if (h->prm.reunit_every > 0)
        for (int j = 0; j < k && j < 40; j++)
            if ((n + j + 1) % h->prm.reunit_every == 0) mask |= 1LL << j;
    if (k > 40) {
        ST(interval_enqueue(h, k, n));
        CU(cudaGetLastError());
        return CULGT_OK;
    }
    long long key = ((mask * 64 + k) << 1) | (h->cur32 ? 1 : 0);
    auto it = h->graphs->exec.find(key);
    if (it == h->graphs->exec.end()) {
        long long before = launches_so_far();
        CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        culgt_status st = interval_enqueue(h, k, n);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
        if (st != CULGT_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return CULGT_ERR_CUDA;
        }
        cudaGraphExec_t exec;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return CULGT_ERR_CUDA;
        }
        int kernels = (int)(launches_so_far() - before);
        count_launch(-kernels);  // captured, not launched
        it = h->graphs->exec.emplace(key, std::make_pair(exec, kernels)).first;
    }
    CU(cudaGraphLaunch(it->second.first, h->stream));
    count_launch(it->second.second);
    return CULGT_OK;
}

// Sweeps the current links until theta < target or the running total n
// reaches max_sweeps; theta is measured first and every check_every sweeps.
// Each check interval is one CUDA graph replay and one host read of theta.
// until_stall (the automatic switch): also stop at the first check, once
// theta < kAutoSwitchFloor, that did not lower theta.
culgt_status run_phase(culgt_handle *h, double target, int *n, int *phase_sweeps, double *theta, double *F,
                       bool until_stall = false)
{
    const culgt_params &p = h->prm;
    ST(theta_now(h, theta, F));
    double prev = INFINITY;
    while (!(*theta < target) && *n < p.max_sweeps) {
        if (until_stall && *theta < kAutoSwitchFloor && !(*theta < prev)) break;
        prev = *theta;
        int k = p.check_every;
        if (k > p.max_sweeps - *n) k = p.max_sweeps - *n;
        ST(run_interval(h, k, *n));
        CU(cudaStreamSynchronize(h->stream));
        CU(cudaGetLastError());
        *n += k;
        *phase_sweeps += k;
        *theta = h->h_scalars[0];
        *F = h->h_scalars[1];
        if (!std::isfinite(*theta) || !std::isfinite(*F)) return CULGT_ERR_NONFINITE;
    }
    return CULGT_OK;
}

culgt_status fix_handle(culgt_handle *h, culgt_result *out)
{
    if (!h->loaded) return CULGT_ERR_ARG;
    const culgt_params &p = h->prm;
    double theta = 0.0, F = 0.0;
    int n = 0;
    h->sweeps32 = h->sweeps64 = 0;
    if ((p.precision == CULGT_MIXED || p.precision == CULGT_MIXED_DF) && h->cur32) {
        if (p.switch_theta > 0.0)
            ST(run_phase(h, p.switch_theta, &n, &h->sweeps32, &theta, &F));
        else
            ST(run_phase(h, p.theta_target, &n, &h->sweeps32, &theta, &F, true));
        ST(culgt_handle_to_fp64(h));
    }
    ST(run_phase(h, p.theta_target, &n, h->cur32 ? &h->sweeps32 : &h->sweeps64, &theta, &F));
    if (out) {
        out->sweeps_fp32 = h->sweeps32;
        out->sweeps_fp64 = h->sweeps64;
        out->theta = theta;
        out->F = F;
    }
    return theta < p.theta_target ? CULGT_OK : CULGT_NOT_CONVERGED;
}

struct HandleGuard {
    culgt_handle *h = nullptr;
    ~HandleGuard() { culgt_destroy(h); }
};

double now_seconds()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// load, (anneal,) fix, diagnostics, store: the body of the one-call entry points
culgt_status fix_call(culgt_handle *h, const void *d_in, void *d_out, culgt_result *out, double t0,
                      const culgt_anneal_params *anneal = nullptr)
{
    culgt_result r;
    std::memset(&r, 0, sizeof r);
    ST(culgt_load(h, d_in));
    ST(plaquette_now(h, &r.plaq_before, h->buf64 != nullptr));
    if (anneal) ST(anneal_now(h, anneal));
    culgt_status st = fix_handle(h, &r);
    if (st < 0) return st;
    ST(plaquette_now(h, &r.plaq_after));
    ST(unitarity_now(h, &r.unitarity_err));
    ST(culgt_store(h, d_out));
    CU(cudaStreamSynchronize(h->stream));
    r.seconds = now_seconds() - t0;
    if (out) *out = r;
    return st;
}

} // namespace

extern "C" {

const char *culgt_status_string(int status)
{
    switch (status) {
    case CULGT_OK: return "CULGT_OK";
    case CULGT_NOT_CONVERGED: return "CULGT_NOT_CONVERGED: max_sweeps reached before theta < theta_target";
    case CULGT_ERR_ARG: return "CULGT_ERR_ARG: invalid argument";
    case CULGT_ERR_DIMS: return "CULGT_ERR_DIMS: every lattice extent must be even and >= 2, V < 2^29";
    case CULGT_ERR_NC: return "CULGT_ERR_NC: nc must be 2 or 3 with a storage_reals valid for it";
    case CULGT_ERR_CUDA: return "CULGT_ERR_CUDA: a CUDA runtime call failed";
    case CULGT_ERR_OOM: return "CULGT_ERR_OOM: device allocation failed";
    case CULGT_ERR_NONFINITE: return "CULGT_ERR_NONFINITE: theta or F is not finite";
    case CULGT_ERR_TIMEOUT: return "CULGT_ERR_TIMEOUT: reserved (no device-side waits in this library)";
    case CULGT_ERR_TOO_LARGE:
        return "CULGT_ERR_TOO_LARGE: lattice above the 4,194,304 sites culgt_theta_static_scratch supports";
    default: return "unknown culgt status";
    }
}

culgt_status culgt_default_params(int nc, const int dims[4], culgt_params *out)
{
    if (!out || !dims) return CULGT_ERR_ARG;
    std::memset(out, 0, sizeof *out);
    for (int mu = 0; mu < 4; mu++) out->dims[mu] = dims[mu];
    out->nc = nc;
    out->omega = 1.7;
    out->or_variant = 0;
    out->precision = CULGT_FP64;
    out->storage_reals = 0;
    out->theta_target = 1e-12;
    out->max_sweeps = 10000;
    out->check_every = 10;
    out->reunit_every = 100;
    out->switch_theta = 1e-8;
    out->dtype_in = 0;
    return validate(out);
}

culgt_status culgt_validate(const culgt_params *p) { return validate(p); }

long long culgt_kernel_launches(void) { return launches_so_far(); }

culgt_status culgt_workspace_bytes(const culgt_params *p, size_t *bytes)
{
    ST(validate(p));
    if (!bytes) return CULGT_ERR_ARG;
    Geom g = make_geom(p->dims);
    const Ops *o32, *o64;
    pick_ops(p, &o32, &o64);
    size_t b = (size_t)max_partials(g) * sizeof(double2) + 4 * sizeof(double);
    if (o32) b += buffer_bytes(o32, g);
    if (o64) b += buffer_bytes(o64, g);
    if (o32 && o64) b += gauge_bytes(o32, g);
    *bytes = b;
    return CULGT_OK;
}

culgt_status culgt_create(const culgt_params *p, void *cuda_stream, culgt_handle **out)
{
    ST(validate(p));
    if (!out) return CULGT_ERR_ARG;
    *out = nullptr;
    culgt_handle *h = new (std::nothrow) culgt_handle;
    if (!h) return CULGT_ERR_OOM;
    std::memset(h, 0, sizeof *h);
    h->prm = *p;
    h->ustream = (cudaStream_t)cuda_stream;
    h->graphs = new (std::nothrow) GraphCache;
    h->geom = make_geom(p->dims);
    pick_ops(p, &h->ops32, &h->ops64);
    h->cur32 = h->ops32 != nullptr;
    culgt_status st = h->graphs ? CULGT_OK : CULGT_ERR_OOM;
    if (st == CULGT_OK && (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess ||
                           cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
                           cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess))
        st = CULGT_ERR_CUDA;
    if (st == CULGT_OK && h->ops32 && cudaMalloc(&h->buf32, buffer_bytes(h->ops32, h->geom)) != cudaSuccess)
        st = CULGT_ERR_OOM;
    if (st == CULGT_OK && h->ops64 && cudaMalloc(&h->buf64, buffer_bytes(h->ops64, h->geom)) != cudaSuccess)
        st = CULGT_ERR_OOM;
    if (st == CULGT_OK && h->ops32 && h->ops64 && cudaMalloc(&h->gacc, gauge_bytes(h->ops32, h->geom)) != cudaSuccess)
        st = CULGT_ERR_OOM;
    if (st == CULGT_OK &&
        cudaMalloc((void **)&h->partials, (size_t)max_partials(h->geom) * sizeof(double2)) != cudaSuccess)
        st = CULGT_ERR_OOM;
    if (st == CULGT_OK && cudaMalloc((void **)&h->d_scalars, 4 * sizeof(double)) != cudaSuccess) st = CULGT_ERR_OOM;
    if (st == CULGT_OK && cudaMallocHost((void **)&h->h_scalars, 4 * sizeof(double)) != cudaSuccess)
        st = CULGT_ERR_OOM;
    if (st != CULGT_OK) {
        (void)cudaGetLastError();
        culgt_destroy(h);
        return st;
    }
    *out = h;
    return CULGT_OK;
}

void culgt_destroy(culgt_handle *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    delete h->graphs;
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->stream) cudaStreamDestroy(h->stream);
    if (h->buf32) cudaFree(h->buf32);
    if (h->buf64) cudaFree(h->buf64);
    if (h->partials) cudaFree(h->partials);
    if (h->d_scalars) cudaFree(h->d_scalars);
    if (h->h_scalars) cudaFreeHost(h->h_scalars);
    if (h->staging) cudaFree(h->staging);
    if (h->gacc) cudaFree(h->gacc);
    delete h;
}

// A mixed handle loads both precisions: the FP32 links it sweeps first and
// the FP64 links the switch rotates by the accumulated g (orbit-exact).
culgt_status culgt_load(culgt_handle *h, const void *d_links)
{
    if (!h || !d_links) return CULGT_ERR_ARG;
    CallScope scope(h);
    const Ops *os[2] = {h->ops32, h->ops64};
    void *bs[2] = {h->buf32, h->buf64};
    for (int k = 0; k < 2; k++) {
        if (!os[k]) continue;
        if (h->prm.dtype_in)
            os[k]->to_internal_f((const float *)d_links, bs[k], h->geom, h->stream);
        else
            os[k]->to_internal_d((const double *)d_links, bs[k], h->geom, h->stream);
    }
    if (h->gacc) h->ops32->gauge_identity(h->gacc, h->geom, h->stream);
    h->cur32 = h->ops32 != nullptr;
    CU(cudaGetLastError());
    h->loaded = 1;
    return CULGT_OK;
}

culgt_status culgt_store(culgt_handle *h, void *d_links)
{
    if (!h || !d_links || !h->loaded) return CULGT_ERR_ARG;
    CallScope scope(h);
    const Ops *o = cur_ops(h);
    if (h->prm.dtype_in)
        o->to_canonical_f(cur_buf(h), (float *)d_links, h->geom, h->stream);
    else
        o->to_canonical_d(cur_buf(h), (double *)d_links, h->geom, h->stream);
    CU(cudaGetLastError());
    return CULGT_OK;
}

culgt_status culgt_handle_sweep(culgt_handle *h, int n_sweeps)
{
    if (!h || !h->loaded || n_sweeps < 0) return CULGT_ERR_ARG;
    CallScope scope(h);
    ST(sweep_now(h, n_sweeps));
    CU(cudaGetLastError());
    return CULGT_OK;
}

culgt_status culgt_handle_theta(culgt_handle *h, double *theta, double *F)
{
    if (!h || !h->loaded) return CULGT_ERR_ARG;
    CallScope scope(h);
    double t, f;
    culgt_status st = theta_now(h, &t, &f);
    if (theta) *theta = t;
    if (F) *F = f;
    return st;
}

culgt_status culgt_handle_plaquette(culgt_handle *h, double *plaq)
{
    if (!h || !h->loaded || !plaq) return CULGT_ERR_ARG;
    CallScope scope(h);
    return plaquette_now(h, plaq);
}

culgt_status culgt_handle_reunitarize(culgt_handle *h)
{
    if (!h || !h->loaded) return CULGT_ERR_ARG;
    CallScope scope(h);
    reunitarize_now(h);
    CU(cudaGetLastError());
    return CULGT_OK;
}

culgt_status culgt_handle_to_fp64(culgt_handle *h)
{
    if (!h || !h->loaded) return CULGT_ERR_ARG;
    CallScope scope(h);
    if (!h->cur32) return CULGT_OK;
    if (!h->ops64) return CULGT_ERR_ARG;  // an FP32-only handle has no FP64 buffer
    if (!h->gacc) return CULGT_ERR_ARG;  // every mixed handle keeps the accumulator
    launch_rotate_orbit(h->ops32, h->gacc, h->ops64, h->buf64, h->geom, h->stream);
    CU(cudaGetLastError());
    h->cur32 = 0;
    return CULGT_OK;
}

culgt_status culgt_handle_tuning(culgt_handle *h, int *threads_per_site, int *block_size, int *min_blocks_per_sm)
{
    if (!h || !h->loaded || !threads_per_site || !block_size || !min_blocks_per_sm) return CULGT_ERR_ARG;
    CallScope scope(h);
    Mapping m;
    ST(tuned_mapping(h, &m));
    *threads_per_site = m.tps;
    *block_size = m.block;
    *min_blocks_per_sm = m.minb;
    return CULGT_OK;
}

culgt_status culgt_handle_fix(culgt_handle *h, culgt_result *out)
{
    if (!h) return CULGT_ERR_ARG;
    CallScope scope(h);
    return fix_handle(h, out);
}

culgt_status culgt_landau_fix(void *d_links, const culgt_params *p, void *cuda_stream, culgt_result *out)
{
    double t0 = now_seconds();
    ST(validate_landau(p));
    if (!d_links) return CULGT_ERR_ARG;
    HandleGuard g;
    ST(culgt_create(p, cuda_stream, &g.h));
    return fix_call(g.h, d_links, d_links, out, t0);
}

culgt_status culgt_mag_fix(void *d_links, const culgt_params *p, void *cuda_stream, culgt_result *out)
{
    double t0 = now_seconds();
    ST(validate(p));
    if (!d_links) return CULGT_ERR_ARG;
    culgt_params q = *p;
    q.gauge = CULGT_MAG;
    HandleGuard g;
    ST(culgt_create(&q, cuda_stream, &g.h));
    return fix_call(g.h, d_links, d_links, out, t0);
}

culgt_status culgt_default_anneal_params(culgt_anneal_params *out)
{
    if (!out) return CULGT_ERR_ARG;
    std::memset(out, 0, sizeof *out);
    out->t_start = 0.6;
    out->t_end = 0.01;
    out->steps = 500;
    out->micro_sweeps = 3;
    out->seed = 0;
    return CULGT_OK;
}

culgt_status culgt_validate_anneal(const culgt_anneal_params *a) { return validate_anneal(a); }

culgt_status culgt_handle_heatbath(culgt_handle *h, double T, unsigned long long seed, unsigned sweep_word)
{
    if (!h || !h->loaded || !(T > 0.0) || std::isinf(T)) return CULGT_ERR_ARG;
    CallScope scope(h);
    ST(heatbath_now(h, T, seed, sweep_word));
    CU(cudaGetLastError());
    return CULGT_OK;
}

culgt_status culgt_handle_heatbath_tuning(culgt_handle *h, int *keep_links, int *min_blocks_per_sm)
{
    if (!h || !h->loaded || !keep_links || !min_blocks_per_sm || h->prm.gauge != CULGT_LANDAU) return CULGT_ERR_ARG;
    CallScope scope(h);
    int v;
    ST(tuned_heatbath(h, &v));
    cur_ops(h)->heatbath_mapping(v, keep_links, min_blocks_per_sm);
    return CULGT_OK;
}

culgt_status culgt_handle_anneal(culgt_handle *h, const culgt_anneal_params *a)
{
    if (!h || !h->loaded) return CULGT_ERR_ARG;
    ST(validate_anneal(a));
    CallScope scope(h);
    return anneal_now(h, a);
}

culgt_status culgt_landau_fix_anneal(void *d_links, const culgt_params *p, const culgt_anneal_params *a,
                                     void *cuda_stream, culgt_result *out)
{
    double t0 = now_seconds();
    ST(validate_landau(p));
    ST(validate_anneal(a));
    if (!d_links) return CULGT_ERR_ARG;
    HandleGuard g;
    ST(culgt_create(p, cuda_stream, &g.h));
    return fix_call(g.h, d_links, d_links, out, t0, a);
}

culgt_status culgt_mag_fix_anneal(void *d_links, const culgt_params *p, const culgt_anneal_params *a,
                                  void *cuda_stream, culgt_result *out)
{
    double t0 = now_seconds();
    ST(validate(p));
    ST(validate_anneal(a));
    if (!d_links) return CULGT_ERR_ARG;
    culgt_params q = *p;
    q.gauge = CULGT_MAG;
    HandleGuard g;
    ST(culgt_create(&q, cuda_stream, &g.h));
    return fix_call(g.h, d_links, d_links, out, t0, a);
}

culgt_status culgt_landau_fix_host(void *h_links, const culgt_params *p, void *cuda_stream, culgt_result *out)
{
    double t0 = now_seconds();
    ST(validate_landau(p));
    if (!h_links) return CULGT_ERR_ARG;
    HandleGuard g;
    ST(culgt_create(p, cuda_stream, &g.h));
    culgt_handle *h = g.h;
    size_t bytes = canonical_bytes(p, h->geom);
    if (cudaMalloc(&h->staging, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        h->staging = nullptr;
        return CULGT_ERR_OOM;
    }
    CU(cudaMemcpyAsync(h->staging, h_links, bytes, cudaMemcpyHostToDevice, h->stream));
    culgt_status st = fix_call(h, h->staging, h->staging, out, t0);
    if (st < 0) return st;
    CU(cudaMemcpyAsync(h_links, h->staging, bytes, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (out) out->seconds = now_seconds() - t0;
    return st;
}

culgt_status culgt_sweep(void *d_links, const culgt_params *p, int n_sweeps, void *cuda_stream)
{
    ST(validate(p));
    if (!d_links || n_sweeps < 0) return CULGT_ERR_ARG;
    HandleGuard g;
    ST(culgt_create(p, cuda_stream, &g.h));
    ST(culgt_load(g.h, d_links));
    ST(culgt_handle_sweep(g.h, n_sweeps));
    ST(culgt_store(g.h, d_links));
    CU(cudaStreamSynchronize(g.h->stream));
    return CULGT_OK;
}

culgt_status culgt_theta(const void *d_links, const culgt_params *p, void *cuda_stream, double *theta, double *F)
{
    ST(validate(p));
    if (!d_links) return CULGT_ERR_ARG;
    HandleGuard g;
    ST(culgt_create(p, cuda_stream, &g.h));
    ST(culgt_load(g.h, d_links));
    return culgt_handle_theta(g.h, theta, F);
}

culgt_status culgt_plaquette(const void *d_links, const culgt_params *p, void *cuda_stream, double *plaq)
{
    ST(validate(p));
    if (!d_links || !plaq) return CULGT_ERR_ARG;
    HandleGuard g;
    ST(culgt_create(p, cuda_stream, &g.h));
    ST(culgt_load(g.h, d_links));
    return plaquette_now(g.h, plaq);
}

culgt_status culgt_reunitarize(void *d_links, const culgt_params *p, void *cuda_stream)
{
    ST(validate(p));
    if (!d_links) return CULGT_ERR_ARG;
    HandleGuard g;
    ST(culgt_create(p, cuda_stream, &g.h));
    ST(culgt_load(g.h, d_links));
    ST(culgt_handle_reunitarize(g.h));
    ST(culgt_store(g.h, d_links));
    CU(cudaStreamSynchronize(g.h->stream));
    return CULGT_OK;
}

} // extern "C"
