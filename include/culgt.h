/*
 * culgt.h — C ABI of libculgt: lattice Landau and Coulomb gauge fixing by
 * checkerboard overrelaxation on one NVIDIA GB300 (sm_103a).
 *
 * The method is the one of Vogt & Schröck, "cuLGT: Lattice Gauge Fixing on
 * GPUs" (GPUHEP2014), Sec. 2: every site x of one checkerboard parity gathers
 *     K(x) = sum_mu [ U_mu(x) + U_mu(x - mu)^+ ],
 * takes the local maximum g(x) of Re tr[g(x) K(x)] (closed form for SU(2),
 * iterated over SU(2) subgroups for SU(3)), overrelaxes it to g^omega and
 * applies it to the 8 links touching x; black sites, then white sites, make
 * one sweep, iterated until the lattice Landau condition Delta(x) = 0 holds to
 * a given precision theta.
 *
 * Conventions shared by every entry point
 *   dims[4]   L0 = time extent, L1..L3 = spatial extents; every extent even
 *             and >= 2 (the checkerboard needs it), V = L0 L1 L2 L3 < 2^29.
 *   site      i = x1 + L1 (x2 + L2 (x3 + L3 x0)) (x1 fastest, time slowest).
 *   parity    p(x) = (x0 + x1 + x2 + x3) mod 2, black = even, swept first.
 *   links     canonical layout [V][4][Nc][Nc] complex, re/im interleaved,
 *             double (dtype_in = 0) or float (dtype_in = 1), in DEVICE memory
 *             owned by the caller, unless an entry point says "host".
 *   theta     (1/V) sum_x tr[Delta(x) Delta(x)^+],
 *             Delta(x) = sum_mu [A_mu(x) - A_mu(x - mu)],
 *             A_mu = [(U_mu - U_mu^+)/(2i)]_traceless   (Sec. 2, with a g = 1).
 *   F         1/(4 Nc V) sum_x sum_mu Re tr U_mu(x)      (Sec. 2, Landau functional).
 *   Coulomb   each time slice t is its own 3D problem over mu = 1..3, with
 *             theta_t, F_t normalised by V3 = L1 L2 L3 and its own
 *             checkerboard (black = x1 + x2 + x3 even).
 *
 * Beyond the Landau/Coulomb overrelaxation of Sec. 2 the library fixes the
 * maximally Abelian gauge (culgt_gauge, culgt_mag_fix) with the same
 * checkerboard skeleton, and combines either gauge with simulated annealing
 * (culgt_anneal_params and the *_anneal entry points): the two other parts of
 * the paper's cuLGT that it names without formulas; the readings are stated
 * beside those declarations.
 *
 * Errors: every function returns a culgt_status and throws nothing. Arguments
 * are validated before any device work. A CUDA error maps to CULGT_ERR_CUDA;
 * the library never prints. Work is ordered on the caller's stream (NULL =
 * legacy default stream); calls that return scalars (theta, F, results)
 * synchronise that stream before returning.
 */
#ifndef CULGT_H
#define CULGT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CULGT_OK = 0,
    CULGT_NOT_CONVERGED = 1,  /* max_sweeps reached before theta < theta_target */
    CULGT_ERR_ARG = -1,       /* NULL pointer, omega outside [1,2), bad counts ... */
    CULGT_ERR_DIMS = -2,      /* an extent odd or < 2, or V too large */
    CULGT_ERR_NC = -3,        /* nc not 2 or 3, or storage_reals not valid for nc */
    CULGT_ERR_CUDA = -4,      /* a CUDA runtime call failed */
    CULGT_ERR_OOM = -5,       /* device allocation failed */
    CULGT_ERR_NONFINITE = -6, /* theta or F came out NaN/Inf (corrupt links) */
    CULGT_ERR_TIMEOUT = -7,   /* reserved: no kernel of this library waits on another */
    CULGT_ERR_TOO_LARGE = -8  /* lattice larger than culgt_theta_static_scratch's fixed scratch */
} culgt_status;

/* Arithmetic of the sweeps. theta and F are always accumulated in FP64.
 *   CULGT_FP64      IEEE FP64 links and arithmetic.
 *   CULGT_FP32      FP32 links and arithmetic.
 *   CULGT_MIXED     FP32 sweeps to switch_theta, then FP64 sweeps to theta_target.
 *   CULGT_MIXED_DF  FP32 sweeps to switch_theta, then double-float sweeps: links
 *                   kept as pairs of floats (hi + lo, ~48 bits, the size of FP64)
 *                   and arithmetic on the FP32 pipes; theta and F formed in FP64
 *                   from the stored pairs.
 *   CULGT_DF        double-float sweeps throughout. */
typedef enum { CULGT_FP64 = 0, CULGT_FP32 = 1, CULGT_MIXED = 2, CULGT_MIXED_DF = 3, CULGT_DF = 4 } culgt_precision;

/* The gauge functional (culgt_params.gauge).
 *   CULGT_LANDAU  F = 1/(4 Nc V) sum_{x,mu} Re tr U_mu(x) (Sec. 2); theta as
 *                 in the Landau entries below. Coulomb gauge is the same
 *                 functional per time slice (culgt_coulomb_fix).
 *   CULGT_MAG     maximally Abelian gauge, named by the paper (abstract) without
 *                 formulas; our reading: F_MAG = 1/(4 Nc V) sum_{x,mu} sum_a
 *                 |U_mu(x)_aa|^2, maximised site by site over the SU(2)
 *                 subgroups with the same checkerboard overrelaxation, and
 *                 theta_MAG = (1/V) sum_x sum_{i != j} |(X_i - X_j)_ij|^2 with
 *                 X_a(x) = sum_mu [U_mu(x) P_a U_mu(x)^+ + U_mu(x-mu)^+ P_a U_mu(x-mu)],
 *                 P_a the diagonal projectors (theta_MAG = 0 at a stationary
 *                 point of the functional). */
typedef enum { CULGT_LANDAU = 0, CULGT_MAG = 1 } culgt_gauge;

typedef struct {
    int dims[4];         /* L0 (time), L1, L2, L3; all even, >= 2 */
    int nc;              /* 2 = SU(2), 3 = SU(3) */
    double omega;        /* overrelaxation parameter, 1 <= omega < 2 (Sec. 2) */
    int or_variant;      /* g^omega: 0 = binomial series to second order (default), 1 = exact power */
    int precision;       /* culgt_precision */
    int storage_reals;   /* reals per link kept in device memory: SU(3) 18 or 12 (first two rows,
                            third rebuilt, Sec. 3.1), SU(2) 4 (quaternion); 0 = default
                            (SU(3): 18 for FP64, 12 for FP32/mixed phase 1; SU(2): 4) */
    double theta_target; /* stop once theta < theta_target */
    int max_sweeps;      /* total sweep budget (both phases of the mixed schedule) */
    int check_every;     /* theta is measured before the first sweep and every check_every sweeps */
    int reunit_every;    /* reunitarise after sweep n when n % reunit_every == 0; 0 = never */
    double switch_theta; /* mixed: leave the FP32 phase once theta < switch_theta; 0 = automatic:
                            past 1e-8 for as long as every check interval still lowers theta,
                            switching at the first that does not (the FP32 rounding floor) */
    int dtype_in;        /* canonical link buffer element type: 0 = double, 1 = float */
    int threads_per_site; /* half-sweep mapping: 1 or 2 threads per site; 0 = autotune */
    int block_size;       /* half-sweep threads per block: 64, 128 or 256; 0 = autotune */
    int min_blocks_per_sm; /* register limit: 1 = none, 3 or 4 blocks of 128 per SM (at most 168 / 128
                              registers, block_size 128); 0 = autotune */
    int gauge;            /* culgt_gauge: the functional the handle API maximises (0 = Landau) */
} culgt_params;

typedef struct {
    int sweeps_fp32;      /* sweeps done with FP32 links */
    int sweeps_fp64;      /* sweeps done with FP64 links */
    double theta;         /* final theta */
    double F;             /* final functional */
    double plaq_before;   /* average plaquette of the input */
    double plaq_after;    /* average plaquette of the output (gauge invariant: should not move) */
    double unitarity_err; /* max_ab |(U U^+ - 1)_ab| over the output links */
    double seconds;       /* wall time of the call */
} culgt_result;

typedef struct culgt_handle culgt_handle;

/* ---- host-only helpers (no device work) ------------------------------- */

/* Human-readable name of a status code. Never NULL. */
const char *culgt_status_string(int status);

/* Fills *out with the library defaults for an SU(nc) lattice of the given
 * dims (omega 1.7, FP64, theta_target 1e-12, max_sweeps 10000, check_every
 * 10, reunit_every 100, switch_theta 1e-8, dtype_in 0). */
culgt_status culgt_default_params(int nc, const int dims[4], culgt_params *out);

/* Validates a parameter block without touching the device. */
culgt_status culgt_validate(const culgt_params *p);

/* Number of kernels this library has launched in this process so far
 * (diagnostic; counted on the host at each launch). */
long long culgt_kernel_launches(void);

/* Device bytes a handle for these parameters allocates. */
culgt_status culgt_workspace_bytes(const culgt_params *p, size_t *bytes);

/* ---- handle API (the hot loop; internal checkerboard layout) -----------
 * A handle owns the links in the internal checkerboard structure-of-arrays
 * layout (Sec. 3.1: parities split, site index fastest), plus reduction
 * scratch. It is bound to one stream and must not be used from two host
 * threads at once. Its sweeps, theta and fix use the functional p->gauge
 * names (Landau or MAG). */

culgt_status culgt_create(const culgt_params *p, void *cuda_stream, culgt_handle **out);
void culgt_destroy(culgt_handle *h);

/* canonical device buffer -> internal layout of the handle's starting
 * precision (FP32 for CULGT_FP32 and CULGT_MIXED, FP64 otherwise). */
culgt_status culgt_load(culgt_handle *h, const void *d_links);
/* internal layout -> canonical device buffer (dtype_in), current precision. */
culgt_status culgt_store(culgt_handle *h, void *d_links);
/* n_sweeps x (black half-sweep, white half-sweep), no theta, no reunitarisation. */
culgt_status culgt_handle_sweep(culgt_handle *h, int n_sweeps);
/* theta and F of the current links (FP64 accumulation). */
culgt_status culgt_handle_theta(culgt_handle *h, double *theta, double *F);
culgt_status culgt_handle_plaquette(culgt_handle *h, double *plaq);
culgt_status culgt_handle_reunitarize(culgt_handle *h);
/* Switches a mixed handle to FP64. The FP32 phase keeps, per site, the
 * product g(x) of its own updates; the switch reunitarises g in FP64 and
 * sets U_mu(x) = g(x) U0_mu(x) g(x+mu)^+ from the FP64 input U0 loaded by
 * culgt_load, so FP32 rounding never moves the links off the gauge orbit of
 * the input (the plaquette is kept to FP64 rounding). No-op in FP64. */
culgt_status culgt_handle_to_fp64(culgt_handle *h);
/* The half-sweep mapping the handle uses. Unless the parameters fix a single
 * mapping, the first sweep times every allowed one (threads per site, block
 * size, register limit; Sec. 5's autotuner) on a scratch copy of the links
 * and keeps, for this storage and volume in the process, the first in its
 * list within 2% of the fastest. Lattices
 * below 65536 sites take the first allowed mapping untimed. The mappings give
 * bitwise identical links; only their speed differs. */
culgt_status culgt_handle_tuning(culgt_handle *h, int *threads_per_site, int *block_size, int *min_blocks_per_sm);
/* Iterates to theta_target as the precision field says (mixed: FP32 until
 * theta < switch_theta, then FP64). Leaves the result in the handle. */
culgt_status culgt_handle_fix(culgt_handle *h, culgt_result *out);

/* ---- one-call API (allocates and frees a handle inside) ---------------- */

/* Landau gauge fixing of d_links in place. out may be NULL. Returns
 * CULGT_NOT_CONVERGED (with the links still written back) if max_sweeps ran
 * out. This and the other Landau/Coulomb one-call, batched and annealing
 * entry points need p->gauge = CULGT_LANDAU (else CULGT_ERR_ARG). */
culgt_status culgt_landau_fix(void *d_links, const culgt_params *p, void *cuda_stream, culgt_result *out);

/* Same, on a HOST buffer (pageable or pinned): host -> device copy, fix,
 * device -> host copy, all inside the call. */
culgt_status culgt_landau_fix_host(void *h_links, const culgt_params *p, void *cuda_stream, culgt_result *out);

/* Maximally Abelian gauge fixing of d_links in place (CULGT_MAG, whatever
 * p->gauge says): sweeps to theta_MAG < theta_target at the given precision,
 * with the mixed schedule and its orbit-exact switch as for Landau gauge.
 * out->theta and out->F are theta_MAG and F_MAG. */
culgt_status culgt_mag_fix(void *d_links, const culgt_params *p, void *cuda_stream, culgt_result *out);

/* Coulomb gauge fixing in place: one 3D problem per time slice over mu =
 * 1..3, each stopping at its own theta_t < theta_target; the accumulated
 * transformation g(x) then rotates the temporal links once,
 * U_0(x) <- g(x) U_0(x) g(x+0)^+. per_slice receives L0 results (may be NULL).
 * d_gauge, if not NULL, receives g(x) as [V][Nc][Nc] complex double. */
culgt_status culgt_coulomb_fix(void *d_links, const culgt_params *p, void *cuda_stream, culgt_result *per_slice,
                               void *d_gauge);

/* Landau gauge fixing like culgt_landau_fix, also returning the gauge
 * transformation: on return d_links = g(x) U_mu(x) g(x+mu)^+ for the input
 * U and d_gauge = g(x) as [V][Nc][Nc] complex double (canonical site order),
 * e.g. to rotate quark fields or propagators the same way. g is accumulated
 * per site in the precision of each phase (FP32 accumulator in the FP32
 * phase, FP64 or double-float afterwards) and reunitarised with the links. */
culgt_status culgt_landau_fix_gauge(void *d_links, const culgt_params *p, void *cuda_stream, culgt_result *out,
                                    void *d_gauge);

/* Maximally Abelian gauge fixing like culgt_mag_fix (p->gauge is taken as
 * CULGT_MAG), also returning g(x) as culgt_landau_fix_gauge does: on return
 * d_links = g(x) U_mu(x) g(x+mu)^+ for the input U and d_gauge = g(x) as
 * [V][Nc][Nc] complex double in canonical site order (the transformation
 * that diagonalises the links as far as the MAG functional of Sec. 1 asks).
 * Errors as culgt_mag_fix; d_gauge NULL is CULGT_ERR_ARG. */
culgt_status culgt_mag_fix_gauge(void *d_links, const culgt_params *p, void *cuda_stream, culgt_result *out,
                                 void *d_gauge);

/* n_sweeps sweeps of d_links in place at the given precision, for the
 * functional p->gauge names. */
culgt_status culgt_sweep(void *d_links, const culgt_params *p, int n_sweeps, void *cuda_stream);

/* theta and F of d_links for the functional p->gauge names (either pointer may be NULL). */
culgt_status culgt_theta(const void *d_links, const culgt_params *p, void *cuda_stream, double *theta, double *F);

/* theta and F like culgt_theta, for callers that cannot allocate device
 * memory while they run: a host program that has given the whole GPU to its
 * own memory pool (cudaMalloc would fail or fragment that pool), or a
 * stream-ordered loop that cannot take the device-wide synchronisation that
 * cudaMalloc/cudaFree may cause. This call allocates nothing: it reads the
 * canonical links in place and keeps its per-block partial sums in a fixed
 * device array inside the library (256 KB; every GPU that loads the library
 * holds it until the process exits). The paper has no counterpart; it is an
 * interface convenience of this library.
 *   d_links  canonical links (device), as for culgt_theta; theta and F are
 *            formed in FP64 whatever dtype_in is.
 *   d_out    device buffer of two doubles: d_out[0] = theta, d_out[1] = F,
 *            written in stream order (the call does not synchronise).
 * Lattices above 4,194,304 sites return CULGT_ERR_TOO_LARGE before any
 * device work. The first call on a device looks up the array's device
 * address with that device current, and so does the first call after the
 * device's context changed (cudaDeviceReset); make such a call before any
 * stream capture. All calls share the array: calls that overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller. */
culgt_status culgt_theta_static_scratch(const void *d_links, const culgt_params *p, void *cuda_stream,
                                        double *d_out);

/* Average plaquette (1/(6 Nc V)) sum_x sum_{mu<nu} Re tr[U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+]. */
culgt_status culgt_plaquette(const void *d_links, const culgt_params *p, void *cuda_stream, double *plaq);

/* Reunitarisation of d_links in place (SU(3): Gram-Schmidt on rows 0, 1,
 * row 2 = conj(row0 x row1); SU(2): normalised quaternion part). */
culgt_status culgt_reunitarize(void *d_links, const culgt_params *p, void *cuda_stream);

/* ---- batched API: many independent problems, one launch per phase ------
 * Problems may differ in dims; nc, precision, omega, the gauge (Landau or
 * MAG) and the stopping rule come from *common (its dims are ignored). Each
 * problem converges and retires on its own theta. out receives n results
 * (may be NULL). */
typedef struct {
    void *d_links;  /* canonical links of this problem, device, dtype_in of *common */
    int dims[4];
} culgt_problem;

culgt_status culgt_fix_batched(const culgt_problem *problems, int n, const culgt_params *common, void *cuda_stream,
                               culgt_result *out);

/* ---- simulated annealing ------------------------------------------------
 * The paper combines overrelaxation with simulated annealing to aim for the
 * global maximum of F among the local maxima (Gribov copies) of a gauge
 * orbit (abstract, Sec. 1), without printing the method; this is our
 * reading of it. A heat-bath sweep is the checkerboard sweep of Sec. 2 with
 * the maximisation of every SU(2) subgroup replaced by a draw from the
 * weight exp(Re tr[r w] / T) over SU(2) at temperature T (x0 by Creutz's
 * method below alpha = 2 k / T = 2, by Kennedy and Pendleton's above). A
 * microcanonical sweep is overrelaxation at omega = 2, which moves the links
 * along the orbit without changing F. Draws come from Philox4x32-10 keyed by
 * the 64-bit seed, with the counter (canonical site index, sweep word,
 * (attempt << 4) | (subgroup << 1) | kind, 0): the draws of a lattice depend
 * on nothing else (not on the thread mapping or on the batch it is in). */
typedef struct {
    double t_start;          /* temperature of the first heat-bath sweep, finite and > 0 */
    double t_end;            /* temperature of the last, finite and > 0 */
    int steps;               /* heat-bath sweeps, >= 0 */
    int micro_sweeps;        /* microcanonical sweeps after each heat-bath sweep, >= 0 */
    unsigned long long seed; /* Philox key (low word, high word) */
} culgt_anneal_params;

/* Defaults for the synthetic fields of the tests (t_start 0.6, t_end 0.01,
 * 500 steps, 3 microcanonical sweeps, seed 0); the paper gives no schedule,
 * tune it per ensemble. */
culgt_status culgt_default_anneal_params(culgt_anneal_params *out);
culgt_status culgt_validate_anneal(const culgt_anneal_params *a);

/* One heat-bath sweep (black, then white) of a loaded handle at temperature
 * T > 0, drawing with the given seed and sweep word. In the FP32 phase of a
 * mixed handle it also accumulates g(x), like an overrelaxation sweep. For a
 * CULGT_MAG handle each subgroup draws B = C Bmax (Bmax the MAG maximiser)
 * with the block functional |z| (2u - 1), u = c0^2 + c3^2, from
 * exp(functional / T): u by exact inversion, the two residual angles
 * uniformly (counter (site, sweep, subgroup << 1, 0)); its microcanonical
 * sweeps are MAG overrelaxation at omega = 2. */
culgt_status culgt_handle_heatbath(culgt_handle *h, double T, unsigned long long seed, unsigned sweep_word);

/* The heat-bath mapping the handle uses: whether the eight links stay in
 * registers between gather and update, and the blocks of 128 per SM the
 * registers are capped for. Chosen like the half-sweep mapping (timed on a
 * scratch copy at the first heat-bath sweep for lattices of 65536 sites and
 * more, cached per storage and volume); every mapping gives the same links. */
culgt_status culgt_handle_heatbath_tuning(culgt_handle *h, int *keep_links, int *min_blocks_per_sm);
/* (CULGT_LANDAU handles; a MAG handle's heat bath has one mapping.) */

/* The annealing schedule on a loaded handle: step k = 0 .. steps-1 is one
 * heat-bath sweep at T_k = t_start + (t_end - t_start) k / (steps - 1)
 * (T_0 = t_start when steps = 1) with sweep word k, then micro_sweeps
 * microcanonical sweeps; counting the sweeps of both kinds, the links are
 * reunitarised after every reunit_every-th. These sweeps are not counted in
 * culgt_result. */
culgt_status culgt_handle_anneal(culgt_handle *h, const culgt_anneal_params *a);

/* Landau gauge fixing like culgt_landau_fix, with the annealing schedule run
 * between the load and the overrelaxation. */
culgt_status culgt_landau_fix_anneal(void *d_links, const culgt_params *p, const culgt_anneal_params *a,
                                     void *cuda_stream, culgt_result *out);

/* Maximally Abelian gauge fixing (culgt_mag_fix) with the annealing
 * schedule run between the load and the overrelaxation. */
culgt_status culgt_mag_fix_anneal(void *d_links, const culgt_params *p, const culgt_anneal_params *a,
                                  void *cuda_stream, culgt_result *out);

/* culgt_fix_batched with the annealing schedule run on every problem first
 * (in shared launches, all problems in step). Problem j draws with the key
 * seed + j, so its draws are those of culgt_landau_fix_anneal (or, with
 * common->gauge = CULGT_MAG, culgt_mag_fix_anneal) with that seed. */
culgt_status culgt_fix_batched_anneal(const culgt_problem *problems, int n, const culgt_params *common,
                                      const culgt_anneal_params *a, void *cuda_stream, culgt_result *out);

/* culgt_coulomb_fix with the annealing schedule run on every time slice
 * first (spatial links, the slice's own checkerboard, g accumulated for the
 * temporal links), all slices in step in shared launches; slice t draws
 * with the key seed + t. */
culgt_status culgt_coulomb_fix_anneal(void *d_links, const culgt_params *p, const culgt_anneal_params *a,
                                      void *cuda_stream, culgt_result *per_slice, void *d_gauge);

#ifdef __cplusplus
}
#endif

#endif /* CULGT_H */
