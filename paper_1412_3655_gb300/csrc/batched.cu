// Host engine of the batched path and its C entry points:
// culgt_fix_batched (independent Landau problems of any sizes) and
// culgt_coulomb_fix (one problem per time slice of one lattice).
//
// Each check interval (check_every sweeps, then theta, decisions and the
// precision switch) is captured once as a CUDA graph and replayed; the host
// reads the phase table after each replay to see whether any problem is
// still sweeping.
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "../../include/culgt.h"
#include "batched_ops.cuh"

using namespace culgt;

namespace {

#define BCU(call)                           \
    do {                                    \
        if ((call) != cudaSuccess) {        \
            (void)cudaGetLastError();       \
            return CULGT_ERR_CUDA;          \
        }                                   \
    } while (0)

double wall_now()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Lattice {
    Geom g;
    void *links32 = nullptr, *links64 = nullptr, *gacc32 = nullptr, *gacc64 = nullptr;
    const void *canon = nullptr;  // caller's canonical buffer
    void *canon_out = nullptr;
    double plaq_before = 0.0;
};

struct Engine {
    culgt_params cp;
    bool coulomb = false;
    bool want_gauge = false;  // keep g(x) in every phase so that it can be returned
    bool has32 = false, has64 = false, acc32 = false, acc64 = false;
    const Ops *o32 = nullptr, *o64 = nullptr;
    const BPhaseOps *b32 = nullptr, *b64 = nullptr;
    cudaStream_t s = nullptr;
    std::vector<Lattice> lat;
    std::vector<BProb> hp;
    std::vector<void *> allocs;
    BProb *dp = nullptr;
    int *d_sweep_map = nullptr, *d_theta_map = nullptr;
    int n_sweep_tiles = 0, n_theta_tiles = 0;
    double2 *partials = nullptr;
    double *d_scal = nullptr;
    BRule rule;
    std::map<int, std::pair<cudaGraphExec_t, int>> graphs;  // key -> (exec, kernels in it)

    ~Engine()
    {
        for (auto &kv : graphs) cudaGraphExecDestroy(kv.second.first);
        for (void *p : allocs) cudaFree(p);
        if (s) cudaStreamDestroy(s);
    }

    culgt_status alloc(void **p, size_t bytes)
    {
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            *p = nullptr;
            return CULGT_ERR_OOM;
        }
        allocs.push_back(*p);
        return CULGT_OK;
    }

    culgt_status init(const culgt_params *p)
    {
        cp = *p;
        const bool mixed = p->precision == CULGT_MIXED || p->precision == CULGT_MIXED_DF;
        const bool df = p->precision == CULGT_MIXED_DF || p->precision == CULGT_DF;
        has32 = p->precision == CULGT_FP32 || mixed;
        has64 = p->precision != CULGT_FP32;
        int def32 = p->nc == 2 ? 4 : 12, def64 = p->nc == 2 ? 4 : 18;
        if (has32) {
            int sr = p->storage_reals ? p->storage_reals : def32;
            o32 = get_ops(p->nc, 1, sr);
            b32 = get_bops(p->nc, 1, sr);
        }
        if (has64 && df) {
            o64 = get_ops_df(p->nc);
            b64 = get_bops_df(p->nc);
        } else if (has64) {
            int sr = (p->precision == CULGT_FP64 && p->storage_reals) ? p->storage_reals : def64;
            o64 = get_ops(p->nc, 0, sr);
            b64 = get_bops(p->nc, 0, sr);
        }
        if ((has32 && (!o32 || !b32)) || (has64 && (!o64 || !b64))) return CULGT_ERR_NC;
        // accumulators: the mixed FP32 phase (orbit-exact switch) and Coulomb (temporal links)
        acc32 = has32 && (has64 || coulomb || want_gauge);
        acc64 = has64 && (coulomb || want_gauge);
        rule.theta_target = p->theta_target;
        rule.auto_switch = mixed && p->switch_theta == 0.0;
        rule.fp32_target = (mixed && !rule.auto_switch) ? p->switch_theta : p->theta_target;
        rule.fp32_next = mixed ? PH_SWITCH : PH_DONE;
        rule.max_sweeps = p->max_sweeps;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            (void)cudaGetLastError();
            s = nullptr;
            return CULGT_ERR_CUDA;
        }
        return CULGT_OK;
    }

    size_t links_bytes(const Ops *o, const Geom &g) const { return (size_t)8 * o->nchunk * g.stride * o->chunk_bytes; }
    size_t acc_bytes(const BPhaseOps *b, const Geom &g) const
    {
        return (size_t)2 * b->acc_nchunk * g.stride * b->acc_chunk_bytes;
    }

    culgt_status add_lattice(const int *dims, const void *canon)
    {
        Lattice L;
        L.g = make_geom(dims);
        L.canon = canon;
        L.canon_out = (void *)canon;
        culgt_status st = CULGT_OK;
        if (has32 && st == CULGT_OK) st = alloc(&L.links32, links_bytes(o32, L.g));
        if (has64 && st == CULGT_OK) st = alloc(&L.links64, links_bytes(o64, L.g));
        if (acc32 && st == CULGT_OK) st = alloc(&L.gacc32, acc_bytes(b32, L.g));
        if (acc64 && st == CULGT_OK) st = alloc(&L.gacc64, acc_bytes(b64, L.g));
        if (st != CULGT_OK) return st;
        lat.push_back(L);
        return CULGT_OK;
    }

    void add_problem(const Lattice &L, int cb_begin, int n_cb, int par_off, int mu_first)
    {
        BProb b;
        std::memset(&b, 0, sizeof b);
        b.g = L.g;
        b.links32 = L.links32;
        b.links64 = L.links64;
        b.gacc32 = L.gacc32;
        b.gacc64 = L.gacc64;
        b.cb_begin = cb_begin;
        b.n_cb = n_cb;
        b.par_off = par_off;
        b.mu_first = mu_first;
        b.sweep_tile0 = n_sweep_tiles;
        b.n_sweep_tiles = (n_cb + kSweepTile - 1) / kSweepTile;
        n_sweep_tiles += b.n_sweep_tiles;
        b.theta_tile0 = n_theta_tiles;
        b.n_theta_tiles = (2 * n_cb + kThetaTile - 1) / kThetaTile;
        n_theta_tiles += b.n_theta_tiles;
        int dirs = 4 - mu_first;
        b.norm_theta = 1.0 / (2.0 * n_cb);
        b.norm_F = 1.0 / ((double)dirs * cp.nc * 2.0 * n_cb);
        b.phase = has32 ? PH_FP32 : PH_FP64;
        b.theta = b.F = 0.0;
        hp.push_back(b);
    }

    // tile maps, problem table, scratch; canonical -> internal; accumulators = 1
    culgt_status upload()
    {
        std::vector<int> sm(n_sweep_tiles), tm(n_theta_tiles);
        for (size_t i = 0; i < hp.size(); i++) {
            for (int t = 0; t < hp[i].n_sweep_tiles; t++) sm[hp[i].sweep_tile0 + t] = (int)i;
            for (int t = 0; t < hp[i].n_theta_tiles; t++) tm[hp[i].theta_tile0 + t] = (int)i;
        }
        culgt_status st = alloc((void **)&dp, hp.size() * sizeof(BProb));
        if (st == CULGT_OK) st = alloc((void **)&d_sweep_map, sm.size() * sizeof(int));
        if (st == CULGT_OK) st = alloc((void **)&d_theta_map, tm.size() * sizeof(int));
        if (st == CULGT_OK) st = alloc((void **)&partials, (size_t)n_theta_tiles * sizeof(double2));
        if (st == CULGT_OK) st = alloc((void **)&d_scal, 4 * sizeof(double));
        if (st != CULGT_OK) return st;
        BCU(cudaMemcpyAsync(dp, hp.data(), hp.size() * sizeof(BProb), cudaMemcpyHostToDevice, s));
        BCU(cudaMemcpyAsync(d_sweep_map, sm.data(), sm.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        BCU(cudaMemcpyAsync(d_theta_map, tm.data(), tm.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        for (Lattice &L : lat) {
            const Ops *os[2] = {o32, o64};
            void *bs[2] = {L.links32, L.links64};
            for (int k = 0; k < 2; k++) {
                if (!os[k]) continue;
                if (cp.dtype_in)
                    os[k]->to_internal_f((const float *)L.canon, bs[k], L.g, s);
                else
                    os[k]->to_internal_d((const double *)L.canon, bs[k], L.g, s);
            }
            if (L.gacc32) b32->gauge_identity(L.gacc32, L.g, s);
            if (L.gacc64) b64->gauge_identity(L.gacc64, L.g, s);
        }
        BCU(cudaGetLastError());
        return CULGT_OK;
    }

    // theta of every problem in `phase`, then its decision
    void check_phase(int phase, int only_switched, int k)
    {
        const BPhaseOps *b = phase == PH_FP32 ? b32 : b64;
        if (cp.gauge == CULGT_MAG)
            b->mag_theta(dp, d_theta_map, n_theta_tiles, phase, only_switched, partials, s);
        else
            b->theta(dp, d_theta_map, n_theta_tiles, phase, only_switched, partials, s);
        k_b_decide<<<(unsigned)hp.size(), 32, 0, s>>>(dp, partials, phase, only_switched, k, rule);
        count_launch();
    }

    void check(int k)
    {
        if (has32) check_phase(PH_FP32, 0, k);
        if (has64) check_phase(PH_FP64, 0, k);
        if (has32 && has64) {
            b64->rotate(dp, d_theta_map, n_theta_tiles, acc64, s);
            k_b_after_switch<<<(unsigned)((hp.size() + 127) / 128), 128, 0, s>>>(dp, (int)hp.size());
            count_launch();
            check_phase(PH_FP64, 1, 0);
        }
    }

    // one colour of an OR half-sweep (Landau or MAG) over every problem in `phase`
    void sweep_colour(const BPhaseOps *b, int colour, int phase, double omega, int variant, bool acc)
    {
        if (cp.gauge == CULGT_MAG)
            b->mag_sweep(dp, d_sweep_map, n_sweep_tiles, colour, phase, omega, variant, acc, s);
        else
            b->sweep(dp, d_sweep_map, n_sweep_tiles, colour, phase, omega, variant, acc, s);
    }

    // k sweeps starting after sweep n, then the check
    void body(int k, int n)
    {
        for (int j = 0; j < k; j++) {
            for (int colour = 0; colour < 2; colour++) {
                if (has32) sweep_colour(b32, colour, PH_FP32, cp.omega, cp.or_variant, acc32);
                if (has64) sweep_colour(b64, colour, PH_FP64, cp.omega, cp.or_variant, acc64);
            }
            if (cp.reunit_every > 0 && (n + j + 1) % cp.reunit_every == 0) {
                if (has32) b32->reunit(dp, d_theta_map, n_theta_tiles, PH_FP32, acc32, s);
                if (has64) b64->reunit(dp, d_theta_map, n_theta_tiles, PH_FP64, acc64, s);
            }
        }
        check(k);
    }

    // replay (capturing on first use) the graph of body(k, n); key: k and the reunitarisation offsets
    culgt_status run_body(int k, int n)
    {
        int key = k;
        if (cp.reunit_every > 0) {
            int mask = 0;
            for (int j = 0; j < k; j++)
                if ((n + j + 1) % cp.reunit_every == 0) mask |= 1 << (j < 30 ? j : 30);
            key = k * 1000003 + mask;
            if (k > 30) {  // too long to key by offsets: launch directly
                body(k, n);
                BCU(cudaGetLastError());
                return CULGT_OK;
            }
        }
        auto it = graphs.find(key);
        if (it == graphs.end()) {
            long long before = launches_so_far();
            BCU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            body(k, n);
            cudaGraph_t graph;
            BCU(cudaStreamEndCapture(s, &graph));
            cudaGraphExec_t exec;
            cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                return CULGT_ERR_CUDA;
            }
            int kernels = (int)(launches_so_far() - before);
            count_launch(-kernels);  // captured, not launched
            it = graphs.emplace(key, std::make_pair(exec, kernels)).first;
        }
        BCU(cudaGraphLaunch(it->second.first, s));
        count_launch(it->second.second);
        return CULGT_OK;
    }

    culgt_status pull()
    {
        BCU(cudaMemcpyAsync(hp.data(), dp, hp.size() * sizeof(BProb), cudaMemcpyDeviceToHost, s));
        BCU(cudaStreamSynchronize(s));
        BCU(cudaGetLastError());
        return CULGT_OK;
    }

    bool any_sweeping() const
    {
        for (const BProb &b : hp)
            if (b.phase == PH_FP32 || b.phase == PH_FP64) return true;
        return false;
    }

    culgt_status run()
    {
        check(0);
        BCU(cudaGetLastError());
        culgt_status st = pull();
        if (st != CULGT_OK) return st;
        int n = 0;
        while (n < cp.max_sweeps && any_sweeping()) {
            int k = cp.check_every < cp.max_sweeps - n ? cp.check_every : cp.max_sweeps - n;
            st = run_body(k, n);
            if (st != CULGT_OK) return st;
            n += k;
            st = pull();
            if (st != CULGT_OK) return st;
        }
        return CULGT_OK;
    }

    // the annealing schedule on every problem, all in the starting phase
    // (FP32 for FP32 and mixed, accumulating g where that phase does)
    culgt_status anneal(const culgt_anneal_params *a)
    {
        const int phase = has32 ? PH_FP32 : PH_FP64;
        const BPhaseOps *b = has32 ? b32 : b64;
        const bool acc = has32 ? acc32 : acc64;
        long long done = 0;
        for (int k = 0; k < a->steps; k++) {
            const double T =
                a->steps > 1 ? a->t_start + (a->t_end - a->t_start) * (double)k / (double)(a->steps - 1) : a->t_start;
            for (int m = 0; m <= a->micro_sweeps; m++) {
                for (int colour = 0; colour < 2; colour++) {
                    if (m == 0 && cp.gauge == CULGT_MAG)
                        b->mag_heatbath(dp, d_sweep_map, n_sweep_tiles, colour, phase, 1.0 / T, a->seed, (uint32_t)k,
                                        acc, s);
                    else if (m == 0)
                        b->heatbath(dp, d_sweep_map, n_sweep_tiles, colour, phase, 1.0 / T, a->seed, (uint32_t)k, acc,
                                    s);
                    else
                        sweep_colour(b, colour, phase, 2.0, 0, acc);
                }
                done++;
                if (cp.reunit_every > 0 && done % cp.reunit_every == 0)
                    b->reunit(dp, d_theta_map, n_theta_tiles, phase, acc, s);
            }
        }
        BCU(cudaGetLastError());
        return CULGT_OK;
    }

    culgt_status plaquette(const Lattice &L, double *P)
    {
        const Ops *o = has64 ? o64 : o32;
        const void *buf = has64 ? L.links64 : L.links32;
        int nb = o->plaq_partials(buf, L.g, partials_for_lattice(), s);
        launch_finalize2(partials_for_lattice(), nb, 1.0 / (6.0 * cp.nc * L.g.V), 0.0, d_scal, s);
        double h[2];
        BCU(cudaMemcpyAsync(h, d_scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        BCU(cudaStreamSynchronize(s));
        *P = h[0];
        return CULGT_OK;
    }

    culgt_status unitarity(const Lattice &L, double *err)
    {
        const Ops *o = has64 ? o64 : o32;
        const void *buf = has64 ? L.links64 : L.links32;
        int nb = o->unitarity_partials(buf, L.g, partials_for_lattice(), s);
        launch_finalize_max(partials_for_lattice(), nb, d_scal, s);
        double h[2];
        BCU(cudaMemcpyAsync(h, d_scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        BCU(cudaStreamSynchronize(s));
        *err = h[0];
        return CULGT_OK;
    }

    double2 *lattice_partials = nullptr;
    size_t lattice_partials_n = 0;
    double2 *partials_for_lattice() { return lattice_partials; }

    culgt_status alloc_lattice_partials()
    {
        size_t n = 0;
        for (const Lattice &L : lat) {
            size_t m = (size_t)max_partials(L.g);
            if (m > n) n = m;
        }
        lattice_partials_n = n;
        return alloc((void **)&lattice_partials, n * sizeof(double2));
    }

    culgt_status store_all()
    {
        for (Lattice &L : lat) {
            const Ops *o = has64 ? o64 : o32;
            const void *buf = has64 ? L.links64 : L.links32;
            if (cp.dtype_in)
                o->to_canonical_f(buf, (float *)L.canon_out, L.g, s);
            else
                o->to_canonical_d(buf, (double *)L.canon_out, L.g, s);
        }
        BCU(cudaGetLastError());
        BCU(cudaStreamSynchronize(s));
        return CULGT_OK;
    }

    culgt_status status() const
    {
        bool nonfinite = false, maxed = false;
        for (const BProb &b : hp) {
            if (b.phase == PH_NONFINITE) nonfinite = true;
            if (b.phase != PH_DONE) maxed = true;
        }
        if (nonfinite) return CULGT_ERR_NONFINITE;
        return maxed ? CULGT_NOT_CONVERGED : CULGT_OK;
    }
};

#define EST(call)                           \
    do {                                    \
        culgt_status s_ = (call);           \
        if (s_ != CULGT_OK) return s_;      \
    } while (0)

} // namespace

namespace {

culgt_status fix_batched(const culgt_problem *problems, int n, const culgt_params *common,
                         const culgt_anneal_params *anneal, void *cuda_stream, culgt_result *out)
{
    double t0 = wall_now();
    if (!problems || n <= 0 || !common) return CULGT_ERR_ARG;
    if (anneal) EST(culgt_validate_anneal(anneal));
    for (int i = 0; i < n; i++) {
        culgt_params p = *common;
        for (int mu = 0; mu < 4; mu++) p.dims[mu] = problems[i].dims[mu];
        culgt_status st = culgt_validate(&p);
        if (st != CULGT_OK) return st;
        if (!problems[i].d_links) return CULGT_ERR_ARG;
    }
    if (cudaStreamSynchronize((cudaStream_t)cuda_stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return CULGT_ERR_CUDA;
    }
    Engine e;
    EST(e.init(common));
    for (int i = 0; i < n; i++) {
        EST(e.add_lattice(problems[i].dims, problems[i].d_links));
        const Geom &g = e.lat.back().g;
        e.add_problem(e.lat.back(), 0, g.Vh, 0, 0);
    }
    EST(e.alloc_lattice_partials());
    EST(e.upload());
    std::vector<double> pb(n), pa(n), ue(n);
    for (int i = 0; i < n; i++) EST(e.plaquette(e.lat[i], &pb[i]));
    if (anneal) EST(e.anneal(anneal));
    EST(e.run());
    for (int i = 0; i < n; i++) {
        EST(e.plaquette(e.lat[i], &pa[i]));
        EST(e.unitarity(e.lat[i], &ue[i]));
    }
    EST(e.store_all());
    double secs = wall_now() - t0;
    if (out)
        for (int i = 0; i < n; i++) {
            const BProb &b = e.hp[i];
            out[i].sweeps_fp32 = b.sweeps32;
            out[i].sweeps_fp64 = b.sweeps64;
            out[i].theta = b.theta;
            out[i].F = b.F;
            out[i].plaq_before = pb[i];
            out[i].plaq_after = pa[i];
            out[i].unitarity_err = ue[i];
            out[i].seconds = secs;
        }
    return e.status();
}

} // namespace

extern "C" culgt_status culgt_fix_batched(const culgt_problem *problems, int n, const culgt_params *common,
                                          void *cuda_stream, culgt_result *out)
{
    return fix_batched(problems, n, common, nullptr, cuda_stream, out);
}

extern "C" culgt_status culgt_fix_batched_anneal(const culgt_problem *problems, int n, const culgt_params *common,
                                                 const culgt_anneal_params *a, void *cuda_stream, culgt_result *out)
{
    if (!a) return CULGT_ERR_ARG;
    return fix_batched(problems, n, common, a, cuda_stream, out);
}

namespace {

// One fix of one lattice in the gauge of p (Landau or MAG) through the
// engine with g(x) kept in every phase, written to d_gauge in the canonical
// order; the input is validated by the callers.
culgt_status fix_gauge_call(void *d_links, const culgt_params *p, void *cuda_stream, culgt_result *out,
                            void *d_gauge, double t0)
{
    if (!d_links || !d_gauge) return CULGT_ERR_ARG;
    if (cudaStreamSynchronize((cudaStream_t)cuda_stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return CULGT_ERR_CUDA;
    }
    Engine e;
    e.want_gauge = true;
    EST(e.init(p));
    EST(e.add_lattice(p->dims, d_links));
    e.add_problem(e.lat[0], 0, e.lat[0].g.Vh, 0, 0);
    EST(e.alloc_lattice_partials());
    EST(e.upload());
    double pb, pa, ue;
    EST(e.plaquette(e.lat[0], &pb));
    EST(e.run());
    EST(e.plaquette(e.lat[0], &pa));
    EST(e.unitarity(e.lat[0], &ue));
    const Lattice &L = e.lat[0];
    const BPhaseOps *b = e.has64 ? e.b64 : e.b32;
    const void *acc = e.has64 ? L.gacc64 : L.gacc32;
    launch_gauge_to_canonical(p->nc, b->fp32 ? 1 : (e.o64->df ? 2 : 0), acc, (double *)d_gauge, L.g, e.s);
    if (cudaGetLastError() != cudaSuccess) return CULGT_ERR_CUDA;
    EST(e.store_all());
    if (out) {
        const BProb &r = e.hp[0];
        out->sweeps_fp32 = r.sweeps32;
        out->sweeps_fp64 = r.sweeps64;
        out->theta = r.theta;
        out->F = r.F;
        out->plaq_before = pb;
        out->plaq_after = pa;
        out->unitarity_err = ue;
        out->seconds = wall_now() - t0;
    }
    return e.status();
}

} // namespace

extern "C" culgt_status culgt_landau_fix_gauge(void *d_links, const culgt_params *p, void *cuda_stream,
                                               culgt_result *out, void *d_gauge)
{
    double t0 = wall_now();
    culgt_status st = culgt_validate(p);
    if (st != CULGT_OK) return st;
    if (p->gauge != CULGT_LANDAU) return CULGT_ERR_ARG;
    return fix_gauge_call(d_links, p, cuda_stream, out, d_gauge, t0);
}

extern "C" culgt_status culgt_mag_fix_gauge(void *d_links, const culgt_params *p, void *cuda_stream,
                                            culgt_result *out, void *d_gauge)
{
    double t0 = wall_now();
    culgt_status st = culgt_validate(p);
    if (st != CULGT_OK) return st;
    culgt_params q = *p;
    q.gauge = CULGT_MAG;
    return fix_gauge_call(d_links, &q, cuda_stream, out, d_gauge, t0);
}

namespace {

culgt_status coulomb_call(void *d_links, const culgt_params *p, const culgt_anneal_params *anneal, void *cuda_stream,
                          culgt_result *per_slice, void *d_gauge)
{
    double t0 = wall_now();
    culgt_status st = culgt_validate(p);
    if (st != CULGT_OK) return st;
    if (p->gauge != CULGT_LANDAU) return CULGT_ERR_ARG;
    if (!d_links) return CULGT_ERR_ARG;
    if (anneal) EST(culgt_validate_anneal(anneal));
    if (cudaStreamSynchronize((cudaStream_t)cuda_stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return CULGT_ERR_CUDA;
    }
    Engine e;
    e.coulomb = true;
    EST(e.init(p));
    EST(e.add_lattice(p->dims, d_links));
    const Lattice &L = e.lat[0];
    const int V3h = L.g.V / p->dims[0] / 2;
    for (int t = 0; t < p->dims[0]; t++) e.add_problem(L, t * V3h, V3h, t & 1, 1);
    EST(e.alloc_lattice_partials());
    EST(e.upload());
    double pb, pa, ue;
    EST(e.plaquette(e.lat[0], &pb));
    if (anneal) EST(e.anneal(anneal));
    EST(e.run());
    // the accumulated g rotates the temporal links (untouched so far)
    if (e.has64)
        e.b64->temporal(L.links64, L.gacc64, L.g, e.s);
    else
        e.b32->temporal(L.links32, L.gacc32, L.g, e.s);
    if (cudaGetLastError() != cudaSuccess) return CULGT_ERR_CUDA;
    EST(e.plaquette(e.lat[0], &pa));
    EST(e.unitarity(e.lat[0], &ue));
    if (d_gauge) {
        // g(x) as [V][Nc][Nc] complex double in canonical site order
        const BPhaseOps *b = e.has64 ? e.b64 : e.b32;
        const void *acc = e.has64 ? L.gacc64 : L.gacc32;
        launch_gauge_to_canonical(p->nc, b->fp32 ? 1 : (e.o64->df ? 2 : 0), acc, (double *)d_gauge, L.g, e.s);
        if (cudaGetLastError() != cudaSuccess) return CULGT_ERR_CUDA;
    }
    EST(e.store_all());
    double secs = wall_now() - t0;
    if (per_slice)
        for (int t = 0; t < p->dims[0]; t++) {
            const BProb &b = e.hp[t];
            per_slice[t].sweeps_fp32 = b.sweeps32;
            per_slice[t].sweeps_fp64 = b.sweeps64;
            per_slice[t].theta = b.theta;
            per_slice[t].F = b.F;
            per_slice[t].plaq_before = pb;
            per_slice[t].plaq_after = pa;
            per_slice[t].unitarity_err = ue;
            per_slice[t].seconds = secs;
        }
    return e.status();
}

} // namespace

extern "C" culgt_status culgt_coulomb_fix(void *d_links, const culgt_params *p, void *cuda_stream,
                                          culgt_result *per_slice, void *d_gauge)
{
    return coulomb_call(d_links, p, nullptr, cuda_stream, per_slice, d_gauge);
}

extern "C" culgt_status culgt_coulomb_fix_anneal(void *d_links, const culgt_params *p, const culgt_anneal_params *a,
                                                 void *cuda_stream, culgt_result *per_slice, void *d_gauge)
{
    if (!a) return CULGT_ERR_ARG;
    return coulomb_call(d_links, p, a, cuda_stream, per_slice, d_gauge);
}
