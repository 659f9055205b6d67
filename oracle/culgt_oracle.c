/*
 * culgt oracle — a plain, slow, obviously-correct FP64 CPU restatement of
 * lattice Landau (and Coulomb) gauge fixing by checkerboard overrelaxation,
 * following Vogt & Schröck, "cuLGT: Lattice Gauge Fixing on GPUs"
 * (GPUHEP2014), Sec. 2 "Lattice Gauge Fixing".
 *
 * TEST INFRASTRUCTURE ONLY. This file is the independent reference the CUDA
 * library is checked against. Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load it. It shares no code, header, table
 * or helper with the CUDA path, and the CUDA path never calls it.
 *
 * Every function is pinned by tests in tests/test_oracle_pins.py against
 * closed forms, brute force and invariants (see the header of each test).
 *
 * Conventions (the paper fixes none of them):
 *   - dims L[0..3]; mu = 0 is time, mu = 1..3 are space; V = L0 L1 L2 L3.
 *   - canonical site index i = x1 + L1 (x2 + L2 (x3 + L3 x0)).
 *   - parity p(x) = (x0 + x1 + x2 + x3) mod 2; "black" = even, swept first.
 *   - link buffer: double[V][4][Nc][Nc][2] (complex, re/im interleaved).
 *   - an SU(2) element is carried as a 2x2 complex matrix everywhere here.
 *
 * Readings of points the paper leaves open (one line each, also listed in
 * the design notes):
 *   R1  SU(3) iterates the subgroups (0,1),(0,2),(1,2) once each, in that
 *       order, and the running K is left-multiplied by each subgroup update.
 *   R2  A 2x2 block w of K is first projected on its quaternion part
 *       P(w) = (w + s2 conj(w) s2)/2 (s2 = Pauli sigma_2), the only part
 *       Re tr[r w] depends on for r in SU(2); the SU(2) maximum g = K^+/sqrt(det K^+)
 *       is then applied to P(w). For SU(2) itself K is a sum of SU(2) matrices,
 *       so P(K) = K and this is the paper's formula as printed.
 *   R3  g^omega is the second-order truncated binomial series
 *       1 + w (g-1) + w(w-1)/2 (g-1)^2, rescaled back onto SU(2)
 *       (variant 0, default); variant 1 is the exact power.
 *   R4  det P(w) = 0 leaves the subgroup untouched (r = 1).
 *   R5  theta = (1/V) sum_x tr[Delta(x) Delta(x)^+] with a g = 1.
 *   R6  Coulomb: each time slice is an independent 3D Landau problem over
 *       mu = 1..3 with its own checkerboard (black = x1+x2+x3 even); the
 *       accumulated g(x) rotates the temporal links once at the end.
 *   R7  Simulated annealing (named, not specified, by the paper) replaces the
 *       maximisation of each SU(2) subgroup (R1) by a heat-bath draw from
 *       exp(Re tr[r w] / T) over SU(2) at temperature T.
 *   R8  Uniforms come from the top 23 bits of a Philox4x32-10 word.
 *   R9  Draw counters: (site, heat-bath sweep, (attempt << 4) | (subgroup << 1)
 *       | kind, 0), keyed by the 64-bit seed.
 *   R10 x0 = 1 - delta by Creutz's method below alpha = 2, by Kennedy and
 *       Pendleton's above; at most 32 attempts, then delta = 0. 1 - x0^2 is
 *       formed as (1 - x0)(1 + x0) from two separately accurate factors.
 *   R11 Schedule: T linear from t_start to t_end over `steps` heat-bath
 *       sweeps, each followed by n_micro microcanonical sweeps (omega = 2);
 *       reunitarisation counts sweeps of both kinds.
 *   R12 Maximally Abelian gauge (named, not specified, by the paper): the
 *       functional is sum_{x,mu} sum_a |U_mu(x)_aa|^2, normalised by Nd Nc V.
 *   R13 Its SU(2) (subgroup) maximiser is the smallest rotation taking the
 *       vector z of the block of X_i - X_j to +|z| e3.
 *   R14 SU(3): the subgroups of R1, running X_a rotated by every step, each
 *       step overrelaxed as in R3.
 *   R15 theta_MAG = (1/V) sum_x sum_{i != j} |(X_i - X_j)_ij|^2.
 *   R16 MAG annealing: each subgroup draws B = C Bmax with u = c0^2 + c3^2
 *       exponential on [0, 1] (rate 2|z|/T), the two residual angles uniform;
 *       microcanonical sweeps are MAG overrelaxation at omega = 2.
 *   R17 Coulomb annealing: each time slice runs the schedule of R11 on its
 *       spatial links with its own checkerboard, keyed by seed + t, before
 *       its overrelaxation; g accumulates for the temporal rotation.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* complex numbers and small matrices                                  */
/* ------------------------------------------------------------------ */

typedef struct { double re, im; } cplx;

static cplx c_make(double re, double im) { cplx z; z.re = re; z.im = im; return z; }
static cplx c_add(cplx a, cplx b) { return c_make(a.re + b.re, a.im + b.im); }
static cplx c_sub(cplx a, cplx b) { return c_make(a.re - b.re, a.im - b.im); }
static cplx c_mul(cplx a, cplx b) { return c_make(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
static cplx c_conj(cplx a) { return c_make(a.re, -a.im); }
static cplx c_scale(cplx a, double s) { return c_make(a.re * s, a.im * s); }
static double c_abs2(cplx a) { return a.re * a.re + a.im * a.im; }
static cplx c_div(cplx a, cplx b)
{
    double d = c_abs2(b);
    return c_scale(c_mul(a, c_conj(b)), 1.0 / d);
}
/* principal square root */
static cplx c_sqrt(cplx z)
{
    double r = sqrt(c_abs2(z));
    double re = sqrt(0.5 * (r + z.re));
    double im = sqrt(0.5 * (r - z.re));
    if (z.im < 0) im = -im;
    return c_make(re, im);
}

/* n x n complex matrix, n = Nc in {2,3} (SU(2) uses the top-left 2x2). */
typedef struct { int n; cplx m[3][3]; } mat;

static mat mat_zero(int n)
{
    mat A;
    memset(&A, 0, sizeof A);
    A.n = n;
    return A;
}
static mat mat_identity(int n)
{
    mat A = mat_zero(n);
    for (int a = 0; a < n; a++) A.m[a][a] = c_make(1.0, 0.0);
    return A;
}
static mat mat_mul(const mat *A, const mat *B)
{
    mat C = mat_zero(A->n);
    for (int a = 0; a < A->n; a++)
        for (int b = 0; b < A->n; b++) {
            cplx s = c_make(0.0, 0.0);
            for (int k = 0; k < A->n; k++) s = c_add(s, c_mul(A->m[a][k], B->m[k][b]));
            C.m[a][b] = s;
        }
    return C;
}
static mat mat_adj(const mat *A)
{
    mat C = mat_zero(A->n);
    for (int a = 0; a < A->n; a++)
        for (int b = 0; b < A->n; b++) C.m[a][b] = c_conj(A->m[b][a]);
    return C;
}
static mat mat_add(const mat *A, const mat *B)
{
    mat C = mat_zero(A->n);
    for (int a = 0; a < A->n; a++)
        for (int b = 0; b < A->n; b++) C.m[a][b] = c_add(A->m[a][b], B->m[a][b]);
    return C;
}
static mat mat_sub(const mat *A, const mat *B)
{
    mat C = mat_zero(A->n);
    for (int a = 0; a < A->n; a++)
        for (int b = 0; b < A->n; b++) C.m[a][b] = c_sub(A->m[a][b], B->m[a][b]);
    return C;
}
static mat mat_scale(const mat *A, cplx s)
{
    mat C = mat_zero(A->n);
    for (int a = 0; a < A->n; a++)
        for (int b = 0; b < A->n; b++) C.m[a][b] = c_mul(A->m[a][b], s);
    return C;
}
static cplx mat_trace(const mat *A)
{
    cplx s = c_make(0.0, 0.0);
    for (int a = 0; a < A->n; a++) s = c_add(s, A->m[a][a]);
    return s;
}
static cplx mat_det2(const mat *A)
{
    return c_sub(c_mul(A->m[0][0], A->m[1][1]), c_mul(A->m[0][1], A->m[1][0]));
}

/* ------------------------------------------------------------------ */
/* lattice geometry                                                    */
/* ------------------------------------------------------------------ */

typedef struct { int L[4]; long V; } lattice;

static lattice make_lattice(const int *L)
{
    lattice lat;
    for (int mu = 0; mu < 4; mu++) lat.L[mu] = L[mu];
    lat.V = (long)L[0] * L[1] * L[2] * L[3];
    return lat;
}
static void site_coords(const lattice *lat, long i, int x[4])
{
    x[1] = (int)(i % lat->L[1]); i /= lat->L[1];
    x[2] = (int)(i % lat->L[2]); i /= lat->L[2];
    x[3] = (int)(i % lat->L[3]); i /= lat->L[3];
    x[0] = (int)i;
}
static long site_index(const lattice *lat, const int x[4])
{
    return x[1] + (long)lat->L[1] * (x[2] + (long)lat->L[2] * (x[3] + (long)lat->L[3] * x[0]));
}
/* the site x + step * mu-hat, periodic */
static long site_shift(const lattice *lat, long i, int mu, int step)
{
    int x[4];
    site_coords(lat, i, x);
    x[mu] = ((x[mu] + step) % lat->L[mu] + lat->L[mu]) % lat->L[mu];
    return site_index(lat, x);
}

static mat get_link(const double *U, int nc, long i, int mu)
{
    mat A = mat_zero(nc);
    const double *p = U + ((size_t)i * 4 + mu) * nc * nc * 2;
    for (int a = 0; a < nc; a++)
        for (int b = 0; b < nc; b++) A.m[a][b] = c_make(p[(a * nc + b) * 2], p[(a * nc + b) * 2 + 1]);
    return A;
}
static void put_link(double *U, int nc, long i, int mu, const mat *A)
{
    double *p = U + ((size_t)i * 4 + mu) * nc * nc * 2;
    for (int a = 0; a < nc; a++)
        for (int b = 0; b < nc; b++) {
            p[(a * nc + b) * 2] = A->m[a][b].re;
            p[(a * nc + b) * 2 + 1] = A->m[a][b].im;
        }
}
static mat get_mat(const double *G, int nc, long k)
{
    mat A = mat_zero(nc);
    const double *p = G + (size_t)k * nc * nc * 2;
    for (int a = 0; a < nc; a++)
        for (int b = 0; b < nc; b++) A.m[a][b] = c_make(p[(a * nc + b) * 2], p[(a * nc + b) * 2 + 1]);
    return A;
}
static void put_mat(double *G, int nc, long k, const mat *A)
{
    double *p = G + (size_t)k * nc * nc * 2;
    for (int a = 0; a < nc; a++)
        for (int b = 0; b < nc; b++) {
            p[(a * nc + b) * 2] = A->m[a][b].re;
            p[(a * nc + b) * 2 + 1] = A->m[a][b].im;
        }
}

/* ------------------------------------------------------------------ */
/* first-order error bounds (for comparing another implementation)     */
/* ------------------------------------------------------------------ */

/* How far one sweep can move each link when its input links and its
 * arithmetic carry small errors. Nothing here changes the sweep; it runs
 * beside it and only sets per-link tolerances when another implementation
 * of the same sweep, rounding differently, is compared with this one. The
 * local problem of Sec. 2 amplifies such differences by the inverse length of
 * the block quaternion it normalises (and the MAG problem by that of the
 * smallest rotation); these bounds say by how much, site by site.
 *
 * Norms: Frobenius for matrices (||.||), Euclidean for quaternions (|.|).
 * Facts used, all to first order in the errors:
 *   F1  a 2x2 block w and its quaternion part a: |da| <= ||dw|| / sqrt2 (the
 *       quaternion part is an orthogonal projection, ||q|| = sqrt2 |a|);
 *   F2  a unit quaternion a/|a| moves by at most |da| / |a|, tangentially
 *       (perpendicular to a);
 *   F3  a change dr of an SU(2) element is |dr| times a unitary 2x2 matrix
 *       (the quaternion matrix of dr / |dr|), so in a 3x3 embedding R
 *       ||dR|| = sqrt2 |dr|, and ||dR K|| = |dr| ||rows i, j of K||;
 *   F4  with unitary factors, ||d(A B)|| <= ||dA|| + ||dB||;
 *   F5  a tangent change of R is dR = dB R with dB in su(2) (rows and columns
 *       i, j), so R X R^+ moves by the commutator [dB, R X R^+], which the
 *       multiple of 1 in R X R^+ does not reach: at most 2 |dr| times the
 *       rows i, j of R X R^+ - l 1 for any real l.
 * Each arithmetic step that rounds is charged rho, the unit of the bound. */
typedef struct {
    double *e;     /* per link, V x 4: bound on ||dU_mu(x)||, updated in place */
    double *slack; /* per site, or NULL: smallest decision slack of the heat bath */
    double rho;    /* charge per rounding step */
    int tight;     /* 1: an SU(3) site's g also takes the tangent bound (tangent_dg) */
} bound_ctx;

/* The site maps the tangent bound distinguishes: Landau (the running matrix
 * is K) or MAG (the three X_a), each by overrelaxation or heat bath. */
typedef struct {
    int mag, hb;
    double omega;
    int variant;
    double inv_T; /* heat bath */
    const uint32_t *key;
    uint32_t site, sweep;
} site_map;

static double tangent_dg(const site_map *m, const mat *state, double E, double rho);

typedef struct {
    double E;     /* bound on the error of the running K (Landau) or of each X_a (MAG) */
    double dg;    /* bound on ||dg|| of the site transformation so far */
    double rho;
    double slack; /* smallest decision slack so far (+inf: none) */
} bound_track;

static const double SQRT2 = 1.4142135623730951;

/* One subgroup step whose SU(2) element moves tangentially by `amp` per
 * unit error of the running matrix, plus one rounding charge: the running
 * matrix's error grows by |dr| times `rows` for the tangent part and times
 * `rows_rho` for the rounding (F3: for Landau both are the Frobenius norm of
 * the rows i, j the step rotates; for MAG F5 and twice the rows of X_a), the
 * site transformation's by sqrt2 |dr| (F3, F4). */
static void track_step2(bound_track *bt, double amp, double rows, double rows_rho)
{
    double d = isinf(amp) ? INFINITY : amp * bt->E;
    bt->E += rows * d + rows_rho * bt->rho;
    bt->dg += SQRT2 * (d + bt->rho);
}

static void track_step(bound_track *bt, double amp, double rows) { track_step2(bt, amp, rows, rows); }

/* ||rows i, j of A|| */
static double rows_norm(const mat *A, int i, int j)
{
    double s = 0.0;
    for (int b = 0; b < A->n; b++) s += c_abs2(A->m[i][b]) + c_abs2(A->m[j][b]);
    return sqrt(s);
}

/* Lipschitz factor of r -> r^omega at the unit quaternion r (R3) for
 * changes dr tangent to the unit sphere (F2). Variant 0: r^omega = v / |v|
 * with v = (1 - omega) e0 + beta(c0) r, beta = omega (1 + (omega - 1)(c0 - 1)),
 * so dv = beta dr + omega (omega - 1) dc0 r, the two terms perpendicular, with
 * |dc0| <= sqrt(1 - c0^2) |dr| for tangent dr; v / |v| moves by at most
 * |dv| / |v|. Variant 1: (cos(omega phi), n sin(omega phi)) moves by omega per
 * unit of phi and by |sin(omega phi)| / sin(phi) per unit of the axis n. */
static double or_lipschitz(const mat *r, double omega, int variant)
{
    double c0 = 0.5 * mat_trace(r).re;
    double n2 = 0.5 * (c_abs2(r->m[0][0]) + c_abs2(r->m[0][1]) + c_abs2(r->m[1][0]) + c_abs2(r->m[1][1]));
    double s = sqrt(fmax(n2 - c0 * c0, 0.0));
    if (variant == 0) {
        double beta = omega * (1.0 + (omega - 1.0) * (c0 - 1.0));
        double v0 = (1.0 - omega) + beta * c0;
        double nv = sqrt(v0 * v0 + beta * beta * s * s);
        double t = omega * (omega - 1.0) * s;
        return nv > 0.0 ? sqrt(beta * beta + t * t) / nv : INFINITY;
    }
    if (!(s > 0.0)) return c0 > 0.0 ? omega : INFINITY;
    return fmax(omega, fabs(sin(omega * atan2(s, c0))) / s);
}

/* ------------------------------------------------------------------ */
/* local maximisation, Sec. 2                                          */
/* ------------------------------------------------------------------ */

/* Quaternion (real-SU(2)-span) part of a 2x2 complex matrix:
 * P(w) = (w + s2 conj(w) s2)/2, where s2 conj(w) s2 = [[w11*, -w10*], [-w01*, w00*]].
 * For r in SU(2), Re tr[r w] = Re tr[r P(w)]  (reading R2). */
static mat su2_part(const mat *w)
{
    mat t = mat_zero(2);
    t.m[0][0] = c_conj(w->m[1][1]);
    t.m[0][1] = c_scale(c_conj(w->m[1][0]), -1.0);
    t.m[1][0] = c_scale(c_conj(w->m[0][1]), -1.0);
    t.m[1][1] = c_conj(w->m[0][0]);
    mat s = mat_add(w, &t);
    return mat_scale(&s, c_make(0.5, 0.0));
}

/* SU(2) local maximum of Re tr[g K]: g = K^+ / sqrt(det K^+)  (Sec. 2),
 * applied to the quaternion part of K (R2); det = 0 gives g = 1 (R4). */
static mat su2_local_max(const mat *K)
{
    mat q = su2_part(K);
    mat qd = mat_adj(&q);
    cplx d = mat_det2(&qd);
    if (d.re == 0.0 && d.im == 0.0) return mat_identity(2);
    cplx s = c_sqrt(d);
    mat g = mat_zero(2);
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) g.m[a][b] = c_div(qd.m[a][b], s);
    return g;
}

/* Overrelaxation g -> g^omega, omega in [1,2)  (Sec. 2, reading R3). */
static mat overrelax(const mat *g, double omega, int variant)
{
    if (variant == 0) {
        /* 1 + w (g-1) + w(w-1)/2 (g-1)^2, then back onto SU(2): the sum is a
         * real multiple of an SU(2) matrix, so divide by sqrt(det). */
        mat one = mat_identity(2);
        mat D = mat_sub(g, &one);
        mat D2 = mat_mul(&D, &D);
        mat t1 = mat_scale(&D, c_make(omega, 0.0));
        mat t2 = mat_scale(&D2, c_make(0.5 * omega * (omega - 1.0), 0.0));
        mat G = mat_add(&one, &t1);
        G = mat_add(&G, &t2);
        cplx s = c_sqrt(mat_det2(&G));
        mat out = mat_zero(2);
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) out.m[a][b] = c_div(G.m[a][b], s);
        return out;
    } else {
        /* exact power: g = cos(phi) 1 + S with S = (g - g^+)/2 = i sin(phi) n.sigma,
         * g^omega = cos(omega phi) 1 + sin(omega phi)/sin(phi) S. */
        mat gd = mat_adj(g);
        mat S = mat_sub(g, &gd);
        S = mat_scale(&S, c_make(0.5, 0.0));
        double cphi = 0.5 * mat_trace(g).re;
        double sphi = sqrt(fmax(mat_det2(&S).re, 0.0));
        if (sphi == 0.0) return *g;
        double phi = atan2(sphi, cphi);
        mat out = mat_scale(&S, c_make(sin(omega * phi) / sphi, 0.0));
        out.m[0][0] = c_add(out.m[0][0], c_make(cos(omega * phi), 0.0));
        out.m[1][1] = c_add(out.m[1][1], c_make(cos(omega * phi), 0.0));
        return out;
    }
}

/* |a| of the quaternion part of a 2x2 block: sqrt(det P(w)) */
static double block_norm(const mat *w)
{
    mat q = su2_part(w);
    return sqrt(fmax(mat_det2(&q).re, 0.0));
}

/* The overrelaxed local gauge transformation g(x) for the gathered K(x).
 * SU(2): g = (K^+/sqrt(det K^+))^omega.  SU(3): iterate over the SU(2)
 * subgroups (R1), each hit maximising Re tr[r w] on its 2x2 block of the
 * running K and then overrelaxed. bt (or NULL) tracks the error bound: the
 * maximiser moves by |da| / |a| <= E / (sqrt2 |a|) (F1, F2), times the
 * overrelaxation's Lipschitz factor. */
static mat local_gauge_b(const mat *K, double omega, int variant, bound_track *bt)
{
    int n = K->n;
    if (n == 2) {
        mat r = su2_local_max(K);
        if (bt) track_step(bt, or_lipschitz(&r, omega, variant) / (SQRT2 * block_norm(K)), 0.0);
        return overrelax(&r, omega, variant);
    }
    static const int sub[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    mat Kr = *K;
    mat g = mat_identity(3);
    for (int s = 0; s < 3; s++) {
        int i = sub[s][0], j = sub[s][1];
        mat w = mat_zero(2);
        w.m[0][0] = Kr.m[i][i];
        w.m[0][1] = Kr.m[i][j];
        w.m[1][0] = Kr.m[j][i];
        w.m[1][1] = Kr.m[j][j];
        mat r = su2_local_max(&w);
        if (bt) track_step(bt, or_lipschitz(&r, omega, variant) / (SQRT2 * block_norm(&w)), rows_norm(&Kr, i, j));
        r = overrelax(&r, omega, variant);
        mat R = mat_identity(3);
        R.m[i][i] = r.m[0][0];
        R.m[i][j] = r.m[0][1];
        R.m[j][i] = r.m[1][0];
        R.m[j][j] = r.m[1][1];
        Kr = mat_mul(&R, &Kr);
        g = mat_mul(&R, &g);
    }
    return g;
}

static mat local_gauge(const mat *K, double omega, int variant) { return local_gauge_b(K, omega, variant, NULL); }

/* ------------------------------------------------------------------ */
/* the checkerboard sweep, Sec. 2                                      */
/* ------------------------------------------------------------------ */

/* K(x) = sum_mu [U_mu(x) + U_mu(x - mu)^+]  over mu = mu_first..3 */
static mat gather_K(const double *U, const lattice *lat, int nc, long i, int mu_first)
{
    mat K = mat_zero(nc);
    for (int mu = mu_first; mu < 4; mu++) {
        mat f = get_link(U, nc, i, mu);
        mat b = get_link(U, nc, site_shift(lat, i, mu, -1), mu);
        mat bd = mat_adj(&b);
        K = mat_add(&K, &f);
        K = mat_add(&K, &bd);
    }
    return K;
}

/* Error bound of a site's local problem: its running matrix starts with
 * the errors of the 2 (4 - mu_first) links it gathers, times `weight` (1 for
 * K; 2 for each X_a of MAG, whose terms U P U^+ move by twice the link), plus
 * one rounding charge. */
static bound_track track_begin(const bound_ctx *bc, const lattice *lat, long i, int mu_first, double weight)
{
    bound_track bt;
    double s = 0.0;
    for (int mu = mu_first; mu < 4; mu++)
        s += bc->e[(size_t)i * 4 + mu] + bc->e[(size_t)site_shift(lat, i, mu, -1) * 4 + mu];
    bt.E = weight * s + bc->rho;
    bt.dg = 0.0;
    bt.rho = bc->rho;
    bt.slack = INFINITY;
    return bt;
}

/* After the site's update: each of its links moved by at most the error of
 * g plus one rounding (F5); the decision slack is recorded per site. */
static void track_end(const bound_ctx *bc, const bound_track *bt, const lattice *lat, long i, int mu_first)
{
    for (int mu = mu_first; mu < 4; mu++) {
        bc->e[(size_t)i * 4 + mu] += bt->dg + bc->rho;
        bc->e[(size_t)site_shift(lat, i, mu, -1) * 4 + mu] += bt->dg + bc->rho;
    }
    if (bc->slack) bc->slack[i] = bt->slack;
}

/* One site update: U_mu(x) <- g U_mu(x), U_mu(x-mu) <- U_mu(x-mu) g^+,
 * i.e. the gauge transformation of Sec. 2 with g = 1 at every other site.
 * bc (or NULL) carries the error bounds along. */
static void update_site_b(double *U, const lattice *lat, int nc, long i, int mu_first,
                          double omega, int variant, double *gacc, const bound_ctx *bc)
{
    mat K = gather_K(U, lat, nc, i, mu_first);
    bound_track bt;
    if (bc) bt = track_begin(bc, lat, i, mu_first, 1.0);
    double E0 = bc ? bt.E : 0.0;
    mat g = local_gauge_b(&K, omega, variant, bc ? &bt : NULL);
    if (bc && bc->tight && nc == 3) {
        site_map m = {0, 0, omega, variant, 0.0, NULL, 0, 0};
        bt.dg = fmin(bt.dg, tangent_dg(&m, &K, E0, bc->rho));
    }
    mat gd = mat_adj(&g);
    for (int mu = mu_first; mu < 4; mu++) {
        long ib = site_shift(lat, i, mu, -1);
        mat f = get_link(U, nc, i, mu);
        mat b = get_link(U, nc, ib, mu);
        mat fn = mat_mul(&g, &f);
        mat bn = mat_mul(&b, &gd);
        put_link(U, nc, i, mu, &fn);
        put_link(U, nc, ib, mu, &bn);
    }
    if (bc) track_end(bc, &bt, lat, i, mu_first);
    if (gacc) {
        mat a = get_mat(gacc, nc, i);
        mat an = mat_mul(&g, &a);
        put_mat(gacc, nc, i, &an);
    }
}

static void update_site(double *U, const lattice *lat, int nc, long i, int mu_first,
                        double omega, int variant, double *gacc)
{
    update_site_b(U, lat, nc, i, mu_first, omega, variant, gacc, NULL);
}

static int site_parity(const lattice *lat, long i, int mu_first)
{
    int x[4];
    site_coords(lat, i, x);
    int p = x[1] + x[2] + x[3];
    if (mu_first == 0) p += x[0];
    return p & 1;
}

/* Update every site of the given parity. Same-parity sites share no link,
 * so the order (and the thread split) does not change the result. */
void oracle_halfsweep(double *U, const int *L, int nc, int parity, double omega, int variant)
{
    lattice lat = make_lattice(L);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < lat.V; i++)
        if (site_parity(&lat, i, 0) == parity) update_site(U, &lat, nc, i, 0, omega, variant, NULL);
}

/* One sweep = black (even) half-sweep, then white (odd). */
void oracle_sweep(double *U, const int *L, int nc, double omega, int variant, int n_sweeps)
{
    for (int s = 0; s < n_sweeps; s++) {
        oracle_halfsweep(U, L, nc, 0, omega, variant);
        oracle_halfsweep(U, L, nc, 1, omega, variant);
    }
}

/* One sweep, exactly as oracle_sweep, carrying the first-order error bounds
 * along: e (V x 4) holds a bound on each input link's error on entry and on
 * each output link's on return, in units of rho (the charge per rounding
 * step; rho = 0 propagates the input errors alone). tight = 1 bounds each
 * SU(3) site's g also by its tangent map (tangent_dg) and keeps the smaller. */
void oracle_sweep_bound(double *U, const int *L, int nc, double omega, int variant, double rho, double *e, int tight)
{
    lattice lat = make_lattice(L);
    bound_ctx bc = {e, NULL, rho, tight};
    for (int parity = 0; parity < 2; parity++) {
#pragma omp parallel for schedule(static)
        for (long i = 0; i < lat.V; i++)
            if (site_parity(&lat, i, 0) == parity) update_site_b(U, &lat, nc, i, 0, omega, variant, NULL, &bc);
    }
}

/* ------------------------------------------------------------------ */
/* gauge precision theta and functional F, Sec. 2                      */
/* ------------------------------------------------------------------ */

/* A_mu(x) = [(U - U^+)/(2i)]_traceless   (a g = 1) */
static mat gauge_field(const mat *U)
{
    int n = U->n;
    mat Ud = mat_adj(U);
    mat D = mat_sub(U, &Ud);
    mat A = mat_scale(&D, c_make(0.0, -0.5)); /* 1/(2i) = -i/2 */
    cplx tr = mat_trace(&A);
    for (int a = 0; a < n; a++) A.m[a][a] = c_sub(A.m[a][a], c_scale(tr, 1.0 / n));
    return A;
}

/* tr[Delta(x) Delta(x)^+], Delta(x) = sum_mu (A_mu(x) - A_mu(x - mu)), mu >= mu_first */
static double site_theta(const double *U, const lattice *lat, int nc, long i, int mu_first)
{
    mat Dl = mat_zero(nc);
    for (int mu = mu_first; mu < 4; mu++) {
        mat f = get_link(U, nc, i, mu);
        mat b = get_link(U, nc, site_shift(lat, i, mu, -1), mu);
        mat Af = gauge_field(&f);
        mat Ab = gauge_field(&b);
        Dl = mat_add(&Dl, &Af);
        Dl = mat_sub(&Dl, &Ab);
    }
    mat Dd = mat_adj(&Dl);
    mat P = mat_mul(&Dl, &Dd);
    return mat_trace(&P).re;
}

static double site_F(const double *U, int nc, long i, int mu_first)
{
    double s = 0.0;
    for (int mu = mu_first; mu < 4; mu++) {
        mat f = get_link(U, nc, i, mu);
        s += mat_trace(&f).re;
    }
    return s;
}

/* theta = (1/V) sum_x tr[Delta Delta^+]   (R5)
 * F     = 1/(Nd Nc V) sum_x sum_mu Re tr U_mu(x)   (Sec. 2, on the current links)
 * Per-site values are summed in site order, so the result is deterministic. */
void oracle_theta(const double *U, const int *L, int nc, double *theta, double *F)
{
    lattice lat = make_lattice(L);
    double *th = (double *)malloc(sizeof(double) * lat.V);
    double *ff = (double *)malloc(sizeof(double) * lat.V);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < lat.V; i++) {
        th[i] = site_theta(U, &lat, nc, i, 0);
        ff[i] = site_F(U, nc, i, 0);
    }
    double st = 0.0, sf = 0.0;
    for (long i = 0; i < lat.V; i++) {
        st += th[i];
        sf += ff[i];
    }
    free(th);
    free(ff);
    *theta = st / (double)lat.V;
    *F = sf / (4.0 * nc * (double)lat.V);
}

/* Average plaquette (1/(6 Nc V)) sum_x sum_{mu<nu} Re tr[U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+],
 * gauge invariant under the transformation of Sec. 2. */
double oracle_plaquette(const double *U, const int *L, int nc)
{
    lattice lat = make_lattice(L);
    double *pp = (double *)malloc(sizeof(double) * lat.V);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < lat.V; i++) {
        double s = 0.0;
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++) {
                mat a = get_link(U, nc, i, mu);
                mat b = get_link(U, nc, site_shift(&lat, i, mu, 1), nu);
                mat c = get_link(U, nc, site_shift(&lat, i, nu, 1), mu);
                mat d = get_link(U, nc, i, nu);
                mat cd = mat_adj(&c), dd = mat_adj(&d);
                mat t = mat_mul(&a, &b);
                t = mat_mul(&t, &cd);
                t = mat_mul(&t, &dd);
                s += mat_trace(&t).re;
            }
        pp[i] = s;
    }
    double s = 0.0;
    for (long i = 0; i < lat.V; i++) s += pp[i];
    free(pp);
    return s / (6.0 * nc * (double)lat.V);
}

/* ------------------------------------------------------------------ */
/* reunitarisation and unitarity                                       */
/* ------------------------------------------------------------------ */

/* SU(3): normalise row 0; row 1 -= (row0^+ . row1) row 0, normalise;
 * row 2 = conj(row0 x row1). SU(2): project on the quaternion part, then
 * divide by sqrt(det). Also the reconstruction rule of the 12-real storage
 * (Sec. 3.1: only the first two rows are kept). */
static mat reunitarize_one(const mat *A)
{
    if (A->n == 2) {
        mat q = su2_part(A);
        cplx s = c_sqrt(mat_det2(&q));
        mat out = mat_zero(2);
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) out.m[a][b] = c_div(q.m[a][b], s);
        return out;
    }
    mat R = *A;
    double n0 = 0.0;
    for (int b = 0; b < 3; b++) n0 += c_abs2(R.m[0][b]);
    n0 = 1.0 / sqrt(n0);
    for (int b = 0; b < 3; b++) R.m[0][b] = c_scale(R.m[0][b], n0);
    cplx ip = c_make(0.0, 0.0);
    for (int b = 0; b < 3; b++) ip = c_add(ip, c_mul(c_conj(R.m[0][b]), R.m[1][b]));
    for (int b = 0; b < 3; b++) R.m[1][b] = c_sub(R.m[1][b], c_mul(ip, R.m[0][b]));
    double n1 = 0.0;
    for (int b = 0; b < 3; b++) n1 += c_abs2(R.m[1][b]);
    n1 = 1.0 / sqrt(n1);
    for (int b = 0; b < 3; b++) R.m[1][b] = c_scale(R.m[1][b], n1);
    for (int b = 0; b < 3; b++) {
        int c = (b + 1) % 3, d = (b + 2) % 3;
        R.m[2][b] = c_conj(c_sub(c_mul(R.m[0][c], R.m[1][d]), c_mul(R.m[0][d], R.m[1][c])));
    }
    return R;
}

/* in place, over n_mats consecutive Nc x Nc matrices */
void oracle_reunitarize(double *M, long n_mats, int nc)
{
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n_mats; k++) {
        mat A = get_mat(M, nc, k);
        mat R = reunitarize_one(&A);
        put_mat(M, nc, k, &R);
    }
}

/* max over matrices of max_ab |(A A^+ - 1)_ab| */
double oracle_unitarity_error(const double *M, long n_mats, int nc)
{
    double worst = 0.0;
    for (long k = 0; k < n_mats; k++) {
        mat A = get_mat(M, nc, k);
        mat Ad = mat_adj(&A);
        mat P = mat_mul(&A, &Ad);
        for (int a = 0; a < nc; a++)
            for (int b = 0; b < nc; b++) {
                cplx e = c_sub(P.m[a][b], c_make(a == b ? 1.0 : 0.0, 0.0));
                double v = sqrt(c_abs2(e));
                if (v > worst) worst = v;
            }
    }
    return worst;
}

/* ------------------------------------------------------------------ */
/* the iteration to a given precision, Sec. 2                          */
/* ------------------------------------------------------------------ */

/* Landau gauge fixing: theta is measured before the first sweep and after
 * every check_every sweeps (and at max_sweeps); the loop stops at the first
 * measurement with theta < theta_target, or at max_sweeps. After sweep n the
 * links are reunitarised when reunit_every > 0 and n % reunit_every == 0.
 * Returns 0 if converged, 1 if max_sweeps was reached. */
int oracle_landau_fix(double *U, const int *L, int nc, double omega, int variant, double theta_target,
                      int max_sweeps, int check_every, int reunit_every, int *sweeps_out, double *theta_out,
                      double *F_out)
{
    lattice lat = make_lattice(L);
    double th, F;
    int n = 0;
    oracle_theta(U, L, nc, &th, &F);
    while (!(th < theta_target) && n < max_sweeps) {
        for (int k = 0; k < check_every && n < max_sweeps; k++) {
            oracle_sweep(U, L, nc, omega, variant, 1);
            n++;
            if (reunit_every > 0 && n % reunit_every == 0) oracle_reunitarize(U, lat.V * 4, nc);
        }
        oracle_theta(U, L, nc, &th, &F);
    }
    *sweeps_out = n;
    *theta_out = th;
    *F_out = F;
    return th < theta_target ? 0 : 1;
}

/* ------------------------------------------------------------------ */
/* Coulomb gauge: one 3D Landau problem per time slice (R6)            */
/* ------------------------------------------------------------------ */

static long slice_site(const lattice *lat, int t, long j)
{
    return (long)t * lat->L[1] * lat->L[2] * lat->L[3] + j;
}

/* theta_t and F_t of time slice t: mu = 1..3, V3 = L1 L2 L3 */
void oracle_theta_slice(const double *U, const int *L, int nc, int t, double *theta, double *F)
{
    lattice lat = make_lattice(L);
    long V3 = (long)L[1] * L[2] * L[3];
    double st = 0.0, sf = 0.0;
    for (long j = 0; j < V3; j++) {
        long i = slice_site(&lat, t, j);
        st += site_theta(U, &lat, nc, i, 1);
        sf += site_F(U, nc, i, 1);
    }
    *theta = st / (double)V3;
    *F = sf / (3.0 * nc * (double)V3);
}

static void slice_halfsweep(double *U, const lattice *lat, int nc, int t, int parity, double omega,
                            int variant, double *gacc)
{
    long V3 = (long)lat->L[1] * lat->L[2] * lat->L[3];
#pragma omp parallel for schedule(static)
    for (long j = 0; j < V3; j++) {
        long i = slice_site(lat, t, j);
        if (site_parity(lat, i, 1) == parity) update_site(U, lat, nc, i, 1, omega, variant, gacc);
    }
}

static void slice_reunitarize(double *U, const lattice *lat, int nc, int t, double *gacc)
{
    long V3 = (long)lat->L[1] * lat->L[2] * lat->L[3];
    for (long j = 0; j < V3; j++) {
        long i = slice_site(lat, t, j);
        for (int mu = 1; mu < 4; mu++) {
            mat A = get_link(U, nc, i, mu);
            mat R = reunitarize_one(&A);
            put_link(U, nc, i, mu, &R);
        }
        mat G = get_mat(gacc, nc, i);
        mat R = reunitarize_one(&G);
        put_mat(gacc, nc, i, &R);
    }
}

static void heatbath_site(double *U, const lattice *lat, int nc, long i, int mu_first, double inv_T,
                          const uint32_t *key, uint32_t sweep, double *gacc);

/* Annealing of one time slice before its overrelaxation (the schedule of
 * R11 on the slice's spatial links, with its checkerboard; draws keyed by
 * key_t, g accumulated into gacc). */
static void slice_anneal(double *U, const lattice *lat, int nc, int t, double t_start, double t_end, int steps,
                         int n_micro, const uint32_t *key_t, int reunit_every, double *gacc)
{
    long V3 = (long)lat->L[1] * lat->L[2] * lat->L[3];
    long done = 0;
    for (int k = 0; k < steps; k++) {
        double T = steps > 1 ? t_start + (t_end - t_start) * (double)k / (double)(steps - 1) : t_start;
        double inv_T = 1.0 / T;
        for (int m = 0; m <= n_micro; m++) {
            for (int parity = 0; parity < 2; parity++) {
                if (m == 0) {
#pragma omp parallel for schedule(static)
                    for (long j = 0; j < V3; j++) {
                        long i = slice_site(lat, t, j);
                        if (site_parity(lat, i, 1) == parity)
                            heatbath_site(U, lat, nc, i, 1, inv_T, key_t, (uint32_t)k, gacc);
                    }
                } else {
                    slice_halfsweep(U, lat, nc, t, parity, 2.0, 0, gacc);
                }
            }
            done++;
            if (reunit_every > 0 && done % reunit_every == 0) slice_reunitarize(U, lat, nc, t, gacc);
        }
    }
}

/* Coulomb gauge fixing: every slice t runs the Landau iteration above on its
 * spatial links alone and stops at its own theta_t; the accumulated g(x) then
 * rotates the temporal links, U_0(x) <- g(x) U_0(x) g(x+0)^+. gacc (V Nc Nc
 * complex) receives the accumulated transformation. Per-slice outputs have
 * L[0] entries. With anneal != NULL (t_start, t_end, steps, n_micro) every
 * slice is first annealed, slice t drawing with the key seed + t. Returns 0
 * if every slice converged. */
static int coulomb_run(double *U, const int *L, int nc, double omega, int variant, double theta_target,
                       int max_sweeps, int check_every, int reunit_every, double *gacc, int *sweeps_t,
                       double *theta_t, double *F_t, const double *anneal, uint64_t seed)
{
    lattice lat = make_lattice(L);
    int all_ok = 1;
    for (long i = 0; i < lat.V; i++) {
        mat I = mat_identity(nc);
        put_mat(gacc, nc, i, &I);
    }
    for (int t = 0; t < L[0]; t++) {
        if (anneal) {
            uint64_t kt = seed + (uint64_t)t;
            uint32_t key_t[2] = {(uint32_t)kt, (uint32_t)(kt >> 32)};
            slice_anneal(U, &lat, nc, t, anneal[0], anneal[1], (int)anneal[2], (int)anneal[3], key_t, reunit_every,
                         gacc);
        }
        double th, F;
        int n = 0;
        oracle_theta_slice(U, L, nc, t, &th, &F);
        while (!(th < theta_target) && n < max_sweeps) {
            for (int k = 0; k < check_every && n < max_sweeps; k++) {
                slice_halfsweep(U, &lat, nc, t, 0, omega, variant, gacc);
                slice_halfsweep(U, &lat, nc, t, 1, omega, variant, gacc);
                n++;
                if (reunit_every > 0 && n % reunit_every == 0) slice_reunitarize(U, &lat, nc, t, gacc);
            }
            oracle_theta_slice(U, L, nc, t, &th, &F);
        }
        sweeps_t[t] = n;
        theta_t[t] = th;
        F_t[t] = F;
        if (!(th < theta_target)) all_ok = 0;
    }
    /* temporal links, read only above */
    for (long i = 0; i < lat.V; i++) {
        mat g = get_mat(gacc, nc, i);
        mat gf = get_mat(gacc, nc, site_shift(&lat, i, 0, 1));
        mat gfd = mat_adj(&gf);
        mat u = get_link(U, nc, i, 0);
        mat t = mat_mul(&g, &u);
        t = mat_mul(&t, &gfd);
        put_link(U, nc, i, 0, &t);
    }
    return all_ok ? 0 : 1;
}

int oracle_coulomb_fix(double *U, const int *L, int nc, double omega, int variant, double theta_target,
                       int max_sweeps, int check_every, int reunit_every, double *gacc, int *sweeps_t,
                       double *theta_t, double *F_t)
{
    return coulomb_run(U, L, nc, omega, variant, theta_target, max_sweeps, check_every, reunit_every, gacc,
                       sweeps_t, theta_t, F_t, NULL, 0);
}

/* Coulomb gauge fixing with every slice annealed first (R11 per slice). */
int oracle_coulomb_fix_anneal(double *U, const int *L, int nc, double t_start, double t_end, int steps, int n_micro,
                              const uint32_t *key, double omega, int variant, double theta_target, int max_sweeps,
                              int check_every, int reunit_every, double *gacc, int *sweeps_t, double *theta_t,
                              double *F_t)
{
    double a[4] = {t_start, t_end, (double)steps, (double)n_micro};
    uint64_t seed = (uint64_t)key[0] | ((uint64_t)key[1] << 32);
    return coulomb_run(U, L, nc, omega, variant, theta_target, max_sweeps, check_every, reunit_every, gacc,
                       sweeps_t, theta_t, F_t, a, seed);
}

/* ------------------------------------------------------------------ */
/* simulated annealing (the paper's abstract and Sec. 1; R7-R11)       */
/* ------------------------------------------------------------------ */

/* Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3", SC 2011): ten rounds, each mapping the counter
 * (c0, c1, c2, c3) with the key (k0, k1) to
 *   (hi(B c2) ^ c1 ^ k0, lo(B c2), hi(A c0) ^ c3 ^ k1, lo(A c0)),
 * A = 0xD2511F53, B = 0xCD9E8D57 (32 x 32 -> 64-bit products), and adding
 * the Weyl increments 0x9E3779B9, 0xBB67AE85 to the key between rounds. */
void oracle_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t pa = (uint64_t)0xD2511F53u * c0;
        uint64_t pb = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)pb;
        uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)pa;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* R8: a uniform in (0, 1) from the top 23 bits m of a word, (m + 1/2) 2^-23:
 * odd multiples of 2^-24, every one exact in float and in double. */
static double unit_uniform(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

/* R9: the counter of a draw: (canonical site index, heat-bath sweep index,
 * (attempt << 4) | (subgroup << 1) | kind, 0); kind 0 = the attempt's four
 * uniforms for x0, kind 1 = the direction. Subgroups count 0, 1, 2 in the
 * order of R1 (0 for SU(2)). */
static void draw4(const uint32_t *key, uint32_t site, uint32_t sweep, uint32_t word2, double u[4])
{
    uint32_t ctr[4] = {site, sweep, word2, 0u};
    uint32_t w[4];
    oracle_philox4x32_10(ctr, key, w);
    for (int k = 0; k < 4; k++) u[k] = unit_uniform(w[k]);
}

#define HB_CREUTZ_BELOW 2.0
static const double TWO_PI = 6.283185307179586;
#define HB_MAX_ATTEMPTS 32

/* R10: delta = 1 - x0 and eps = 1 + x0 for an SU(2) element x whose x0 has
 * the density proportional to sqrt(1 - x0^2) exp(alpha x0) on [-1, 1] (the
 * heat-bath distribution of the subgroup at temperature T, alpha = 2 k / T,
 * see below). alpha < 2: Creutz's method, x0 drawn from exp(alpha x0) by
 * inverting its distribution function, kept with probability
 * sqrt(1 - x0^2); the inversion gives delta and eps each from its own
 * logarithm, so that both keep their relative accuracy near x0 = +1 and -1.
 * alpha >= 2: Kennedy and Pendleton's, delta drawn from Gamma(3/2, alpha) as
 * -(log u0 + cos^2(2 pi u1) log u2) / alpha, kept with probability
 * sqrt(1 - delta/2), and eps = 2 - delta. Both tests compare squares, with
 * 1 - x0^2 = delta eps. After HB_MAX_ATTEMPTS rejections (below 1e-16 at any
 * alpha) the draw gives delta = 0, eps = 2. *attempts receives the number of
 * attempts made. */
/* Attempt a of the draw: the candidate delta and eps, and the two sides of
 * its acceptance test (kept when lhs <= rhs). */
static void hb_attempt(double alpha, const uint32_t *key, uint32_t site, uint32_t sweep, int sub, int a,
                       double *delta, double *eps, double *lhs, double *rhs)
{
    double u[4];
    draw4(key, site, sweep, ((uint32_t)a << 4) | ((uint32_t)sub << 1), u);
    if (alpha < HB_CREUTZ_BELOW) {
        double d = -log1p(u[0] * expm1(-2.0 * alpha)) / alpha;
        double e = log1p((1.0 - u[0]) * expm1(2.0 * alpha)) / alpha;
        *delta = d;
        *eps = e;
        *lhs = u[1] * u[1];
        *rhs = d * e;
    } else {
        double c = cos(TWO_PI * u[1]);
        double d = -(log(u[0]) + c * c * log(u[2])) / alpha;
        *delta = d;
        *eps = 2.0 - d;
        *lhs = u[3] * u[3];
        *rhs = 1.0 - 0.5 * d;
    }
}

static void hb_draw(double alpha, const uint32_t *key, uint32_t site, uint32_t sweep, int sub, double *delta,
                    double *eps, int *attempts)
{
    for (int a = 0; a < HB_MAX_ATTEMPTS; a++) {
        double d, e, lhs, rhs;
        hb_attempt(alpha, key, site, sweep, sub, a, &d, &e, &lhs, &rhs);
        if (attempts) *attempts = a + 1;
        if (lhs <= rhs) {
            *delta = d;
            *eps = e;
            return;
        }
    }
    *delta = 0.0;
    *eps = 2.0;
}

/* Relative step of the central differences in alpha (or beta) below: large
 * enough that rounding (1e-16 / 1e-6) stays far below the derivative, small
 * enough that the second-order remainder does too. */
#define FD_STEP 1e-6

/* Error bound of one heat-bath subgroup draw (R7, R10) at alpha = 2 k / T
 * when the block is known to within E (Frobenius). The maximiser v moves by
 * E / (sqrt2 k) (F1, F2); alpha moves by 2 |dk| / T <= sqrt2 E / T, and x with
 * it by |dx/dalpha| per unit (a central difference of the accepted attempt's
 * (delta, sqrt(delta eps)) with the same uniforms); r = x v moves by the sum.
 * A decision whose two sides differ by less than their own error may go the
 * other way in another implementation: for every attempt made, and for the
 * choice of method at alpha = 2, the decision slack is the margin divided by
 * that error (16 rounding charges for the compared values plus the margin's
 * sensitivity to alpha times alpha's error); a slack below the unit roundoff
 * of an implementation marks a decision it may take differently. */
static void hb_track(bound_track *bt, double k, double alpha, double inv_T, const uint32_t *key, uint32_t site,
                     uint32_t sweep, int sub, double rows)
{
    double dalpha = SQRT2 * inv_T * bt->E; /* bound on alpha's error */
    double sl = fabs(alpha - HB_CREUTZ_BELOW) / (4.0 * bt->rho * alpha + dalpha);
    double xprime = 0.0;
    double h = FD_STEP * alpha;
    for (int a = 0; a < HB_MAX_ATTEMPTS; a++) {
        double d, e, lhs, rhs, dp, ep, lp, rp, dm, em, lm, rm;
        hb_attempt(alpha, key, site, sweep, sub, a, &d, &e, &lhs, &rhs);
        hb_attempt(alpha + h, key, site, sweep, sub, a, &dp, &ep, &lp, &rp);
        hb_attempt(alpha - h, key, site, sweep, sub, a, &dm, &em, &lm, &rm);
        double mprime = fabs((lp - rp) - (lm - rm)) / (2.0 * h);
        sl = fmin(sl, fabs(lhs - rhs) / (16.0 * bt->rho + mprime * dalpha));
        if (lhs <= rhs) {
            double dd = (dp - dm) / (2.0 * h);
            double ds = (sqrt(fmax(dp * ep, 0.0)) - sqrt(fmax(dm * em, 0.0))) / (2.0 * h);
            xprime = sqrt(dd * dd + ds * ds);
            break;
        }
    }
    bt->slack = fmin(bt->slack, sl);
    track_step(bt, (1.0 / k + xprime * 2.0 * inv_T) / SQRT2, rows);
}

/* The decision slack of hb_track for one draw whose alpha is known to
 * within dalpha (no rounding charges): below 1, some alpha within dalpha may
 * take one of the draw's decisions the other way. */
double oracle_hb_slack(double alpha, double dalpha, double T, const uint32_t *key, uint32_t site, uint32_t sweep,
                       int sub)
{
    bound_track bt = {dalpha * T / SQRT2, 0.0, 0.0, INFINITY};
    hb_track(&bt, 0.5 * alpha * T, alpha, 1.0 / T, key, site, sweep, sub, 0.0);
    return bt.slack;
}

double oracle_hb_delta(double alpha, const uint32_t *key, uint32_t site, uint32_t sweep, int sub, int *attempts)
{
    double d, e;
    hb_draw(alpha, key, site, sweep, sub, &d, &e, attempts);
    return d;
}

/* The unit quaternion x = (1 - delta, s n) with s = sqrt(delta eps) and n
 * uniform on the sphere: cos(theta) = 2 u0 - 1, sin(theta) = 2 sqrt(u0 (1 - u0)),
 * phi = 2 pi u1. */
void oracle_hb_x(double alpha, const uint32_t *key, uint32_t site, uint32_t sweep, int sub, double *x)
{
    double delta, eps;
    hb_draw(alpha, key, site, sweep, sub, &delta, &eps, NULL);
    double u[4];
    draw4(key, site, sweep, ((uint32_t)sub << 1) | 1u, u);
    double ct = 2.0 * u[0] - 1.0;
    double st = 2.0 * sqrt(u[0] * (1.0 - u[0]));
    double phi = TWO_PI * u[1];
    double s = sqrt(delta * eps);
    x[0] = 1.0 - delta;
    x[1] = s * st * cos(phi);
    x[2] = s * st * sin(phi);
    x[3] = s * ct;
}

/* the 2x2 matrix x0 1 + i (x1 s1 + x2 s2 + x3 s3) */
static mat quaternion_matrix(const double *x)
{
    mat X = mat_zero(2);
    X.m[0][0] = c_make(x[0], x[3]);
    X.m[0][1] = c_make(x[2], x[1]);
    X.m[1][0] = c_make(-x[2], x[1]);
    X.m[1][1] = c_make(x[0], -x[3]);
    return X;
}

/* Heat bath for one 2x2 block w at temperature T (R7): with q = P(w) = k v^+,
 * k = sqrt(det q) and v = q^+/k the maximiser of Re tr[r w], every r = x v
 * has Re tr[r w] = Re tr[x v q] = k Re tr[x] = 2 k x0, so the Boltzmann
 * weight exp(Re tr[r w] / T) over Haar measure is that of x0 above with
 * alpha = 2 k / T and a uniform direction. r = x v, rescaled to det r = 1.
 * k = 0 leaves the block alone (as R4). */
static mat heatbath_su2(const mat *w, double inv_T, const uint32_t *key, uint32_t site, uint32_t sweep, int sub,
                        bound_track *bt, double rows)
{
    mat q = su2_part(w);
    double k = sqrt(mat_det2(&q).re);
    if (!(k > 0.0)) {
        if (bt) track_step(bt, INFINITY, rows);
        return mat_identity(2);
    }
    if (bt) hb_track(bt, k, (2.0 * k) * inv_T, inv_T, key, site, sweep, sub, rows);
    mat v = su2_local_max(w);
    double x[4];
    oracle_hb_x((2.0 * k) * inv_T, key, site, sweep, sub, x);
    mat X = quaternion_matrix(x);
    mat r = mat_mul(&X, &v);
    cplx s = c_sqrt(mat_det2(&r));
    mat out = mat_zero(2);
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) out.m[a][b] = c_div(r.m[a][b], s);
    return out;
}

/* The heat-bath gauge transformation of one site: SU(2) directly, SU(3)
 * over the subgroups of R1 with the running K, as in local_gauge. */
static mat heatbath_gauge(const mat *K, double inv_T, const uint32_t *key, uint32_t site, uint32_t sweep,
                          bound_track *bt)
{
    int n = K->n;
    if (n == 2) return heatbath_su2(K, inv_T, key, site, sweep, 0, bt, 0.0);
    static const int sub[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    mat Kr = *K;
    mat g = mat_identity(3);
    for (int s = 0; s < 3; s++) {
        int i = sub[s][0], j = sub[s][1];
        mat w = mat_zero(2);
        w.m[0][0] = Kr.m[i][i];
        w.m[0][1] = Kr.m[i][j];
        w.m[1][0] = Kr.m[j][i];
        w.m[1][1] = Kr.m[j][j];
        mat r = heatbath_su2(&w, inv_T, key, site, sweep, s, bt, rows_norm(&Kr, i, j));
        mat R = mat_identity(3);
        R.m[i][i] = r.m[0][0];
        R.m[i][j] = r.m[0][1];
        R.m[j][i] = r.m[1][0];
        R.m[j][j] = r.m[1][1];
        Kr = mat_mul(&R, &Kr);
        g = mat_mul(&R, &g);
    }
    return g;
}

static void heatbath_site_b(double *U, const lattice *lat, int nc, long i, int mu_first, double inv_T,
                            const uint32_t *key, uint32_t sweep, double *gacc, const bound_ctx *bc)
{
    mat K = gather_K(U, lat, nc, i, mu_first);
    bound_track bt;
    if (bc) bt = track_begin(bc, lat, i, mu_first, 1.0);
    double E0 = bc ? bt.E : 0.0;
    mat g = heatbath_gauge(&K, inv_T, key, (uint32_t)i, sweep, bc ? &bt : NULL);
    if (bc && bc->tight && nc == 3) {
        site_map m = {0, 1, 0.0, 0, inv_T, key, (uint32_t)i, sweep};
        bt.dg = fmin(bt.dg, tangent_dg(&m, &K, E0, bc->rho));
    }
    mat gd = mat_adj(&g);
    for (int mu = mu_first; mu < 4; mu++) {
        long ib = site_shift(lat, i, mu, -1);
        mat f = get_link(U, nc, i, mu);
        mat b = get_link(U, nc, ib, mu);
        mat fn = mat_mul(&g, &f);
        mat bn = mat_mul(&b, &gd);
        put_link(U, nc, i, mu, &fn);
        put_link(U, nc, ib, mu, &bn);
    }
    if (bc) track_end(bc, &bt, lat, i, mu_first);
    if (gacc) {
        mat a = get_mat(gacc, nc, i);
        mat an = mat_mul(&g, &a);
        put_mat(gacc, nc, i, &an);
    }
}

static void heatbath_site(double *U, const lattice *lat, int nc, long i, int mu_first, double inv_T,
                          const uint32_t *key, uint32_t sweep, double *gacc)
{
    heatbath_site_b(U, lat, nc, i, mu_first, inv_T, key, sweep, gacc, NULL);
}

/* One heat-bath sweep at temperature T (black, then white; Landau, mu =
 * 0..3); `sweep` is the counter word of its draws. gacc (V Nc Nc complex, or
 * NULL) accumulates g(x) <- g(x) gacc(x). */
void oracle_heatbath_halfsweep(double *U, const int *L, int nc, int parity, double T, const uint32_t *key,
                               uint32_t sweep, double *gacc)
{
    lattice lat = make_lattice(L);
    double inv_T = 1.0 / T;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < lat.V; i++)
        if (site_parity(&lat, i, 0) == parity) heatbath_site(U, &lat, nc, i, 0, inv_T, key, sweep, gacc);
}

void oracle_heatbath_sweep(double *U, const int *L, int nc, double T, const uint32_t *key, uint32_t sweep,
                           double *gacc)
{
    oracle_heatbath_halfsweep(U, L, nc, 0, T, key, sweep, gacc);
    oracle_heatbath_halfsweep(U, L, nc, 1, T, key, sweep, gacc);
}

/* One heat-bath sweep, exactly as oracle_heatbath_sweep, with the error
 * bounds of oracle_sweep_bound in e (V x 4) and each site's smallest
 * decision slack in slack (V). */
void oracle_heatbath_sweep_bound(double *U, const int *L, int nc, double T, const uint32_t *key, uint32_t sweep,
                                 double rho, double *e, double *slack, int tight)
{
    lattice lat = make_lattice(L);
    bound_ctx bc = {e, slack, rho, tight};
    double inv_T = 1.0 / T;
    for (int parity = 0; parity < 2; parity++) {
#pragma omp parallel for schedule(static)
        for (long i = 0; i < lat.V; i++)
            if (site_parity(&lat, i, 0) == parity) heatbath_site_b(U, &lat, nc, i, 0, inv_T, key, sweep, NULL, &bc);
    }
}

/* Microcanonical sweep: overrelaxation at omega = 2, r -> r^2 for the
 * maximiser r of every subgroup, which keeps each local functional (R11). */
void oracle_micro_sweep(double *U, const int *L, int nc)
{
    oracle_sweep(U, L, nc, 2.0, 0, 1);
}

/* R11: the annealing schedule. Step k = 0..steps-1 runs one heat-bath sweep
 * at T_k = t_start + (t_end - t_start) k / (steps - 1) (T_0 = t_start for
 * steps = 1) with counter word `sweep` = k, then n_micro microcanonical
 * sweeps. Counting every sweep of either kind, the links are reunitarised
 * after each reunit_every-th (reunit_every > 0). */
void oracle_anneal(double *U, const int *L, int nc, double t_start, double t_end, int steps, int n_micro,
                   const uint32_t *key, int reunit_every)
{
    lattice lat = make_lattice(L);
    long done = 0;
    for (int k = 0; k < steps; k++) {
        double T = steps > 1 ? t_start + (t_end - t_start) * (double)k / (double)(steps - 1) : t_start;
        for (int m = 0; m <= n_micro; m++) {
            if (m == 0)
                oracle_heatbath_sweep(U, L, nc, T, key, (uint32_t)k, NULL);
            else
                oracle_micro_sweep(U, L, nc);
            done++;
            if (reunit_every > 0 && done % reunit_every == 0) oracle_reunitarize(U, lat.V * 4, nc);
        }
    }
}

/* ------------------------------------------------------------------ */
/* maximally Abelian gauge (abstract, Sec. 1; readings R12-R15)        */
/* ------------------------------------------------------------------ */

/* R12: the MAG functional is F_MAG = 1/(Nd Nc V) sum_{x,mu} sum_a |U_mu(x)_aa|^2
 * (1 when every link is diagonal). With the diagonal projectors P_a, the
 * part of it that depends on g(x) is sum_a tr[P_a g X_a g^+] with
 *   X_a(x) = sum_mu [U_mu(x) P_a U_mu(x)^+ + U_mu(x-mu)^+ P_a U_mu(x-mu)],
 * since |(g U)_aa|^2 = tr[P_a g U P_a U^+ g^+] and
 * |(U g^+)_aa|^2 = tr[P_a g U^+ P_a U g^+]. */
static void mag_X(const double *U, const lattice *lat, int nc, long i, mat *X)
{
    for (int a = 0; a < nc; a++) X[a] = mat_zero(nc);
    for (int mu = 0; mu < 4; mu++) {
        mat f = get_link(U, nc, i, mu);
        mat b = get_link(U, nc, site_shift(lat, i, mu, -1), mu);
        mat fd = mat_adj(&f), bd = mat_adj(&b);
        for (int a = 0; a < nc; a++) {
            mat Pa = mat_zero(nc);
            Pa.m[a][a] = c_make(1.0, 0.0);
            mat t = mat_mul(&f, &Pa);
            t = mat_mul(&t, &fd);
            X[a] = mat_add(&X[a], &t);
            t = mat_mul(&bd, &Pa);
            t = mat_mul(&t, &b);
            X[a] = mat_add(&X[a], &t);
        }
    }
}

/* R13: for an SU(2) element B acting on rows and columns (i, j), the
 * g-dependent part of the local functional is (1/2) tr[s3 B Z B^+] + const
 * with Z the (i, j) block of X_i - X_j. Writing the traceless part of Z as
 * z.s, this is (R(B) z)_3, R(B) the rotation B induces; its maximum |z| is
 * reached by the smallest rotation taking z to +|z| e3,
 *   B = (|z| 1 + s3 (z.s)) / sqrt(2 |z| (|z| + z3)).
 * z = 0 leaves the block alone; z = -|z| e3 takes B = i s1. */
static mat mag_su2_max(const mat *Z)
{
    double z3 = 0.5 * (Z->m[0][0].re - Z->m[1][1].re);
    double z1 = Z->m[0][1].re, z2 = -Z->m[0][1].im; /* Z_01 = z1 - i z2 */
    double n = sqrt(z1 * z1 + z2 * z2 + z3 * z3);
    mat B = mat_zero(2);
    if (!(n > 0.0)) return mat_identity(2);
    if (!(n + z3 > 0.0)) { /* z on (or by rounding past) -e3 */
        B.m[0][1] = c_make(0.0, 1.0);
        B.m[1][0] = c_make(0.0, 1.0);
        return B;
    }
    /* s3 (z.s) = [[z3, z1 - i z2], [-(z1 + i z2), z3]] */
    B.m[0][0] = c_make(n + z3, 0.0);
    B.m[0][1] = c_make(z1, -z2);
    B.m[1][0] = c_make(-z1, -z2);
    B.m[1][1] = c_make(n + z3, 0.0);
    cplx s = c_sqrt(mat_det2(&B));
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) B.m[a][b] = c_div(B.m[a][b], s);
    return B;
}

/* R14: the MAG site transformation: SU(2) directly, SU(3) over the subgroups
 * of R1, each maximising its block and overrelaxed (R3), the running X_a
 * rotated by every subgroup update (X_a <- R X_a R^+, g <- R g). */
/* Error bound of the MAG maximiser of a block Z whose X_a are known to
 * within E: z moves by at most ||dZ|| <= 2 E, and the smallest rotation
 * (|z| + z3, -z2, z1, 0) / N, N = sqrt(2 |z| (|z| + z3)), depends on z / |z|
 * alone, so it moves by |dz| / N (an unnormalised vector that moves as
 * z / |z| does, over its length sqrt(2 (1 + z3 / |z|))). Returns 2 / N. */
static double mag_max_amp(const mat *Z)
{
    double z3 = 0.5 * (Z->m[0][0].re - Z->m[1][1].re);
    double z1 = Z->m[0][1].re, z2 = -Z->m[0][1].im;
    double n = sqrt(z1 * z1 + z2 * z2 + z3 * z3);
    double N = sqrt(fmax(2.0 * n * (n + z3), 0.0));
    return N > 0.0 ? 2.0 / N : INFINITY;
}

/* X_a <- R X_a R^+ moves by at most this per unit of |dr|: for a tangent
 * change (shifted = 1) 2 max_a ||rows i, j of X_a - l_a 1|| with l_a the mean
 * of the diagonal entries i, j (F5), for any change 2 max_a ||rows i, j of X_a|| (F3) */
static double mag_rows(const mat *X, int nc, int i, int j, int shifted)
{
    double m = 0.0;
    for (int a = 0; a < nc; a++) {
        mat Y = X[a];
        if (shifted) {
            double l = 0.5 * (X[a].m[i][i].re + X[a].m[j][j].re);
            for (int b = 0; b < nc; b++) Y.m[b][b].re -= l;
        }
        m = fmax(m, rows_norm(&Y, i, j));
    }
    return 2.0 * m;
}

static mat mag_local_gauge_b(mat *X, int nc, double omega, int variant, bound_track *bt)
{
    static const int sub[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    int nsub = nc == 2 ? 1 : 3;
    mat g = mat_identity(nc);
    for (int s = 0; s < nsub; s++) {
        int i = sub[s][0], j = sub[s][1];
        mat D = mat_sub(&X[i], &X[j]);
        mat Z = mat_zero(2);
        Z.m[0][0] = D.m[i][i];
        Z.m[0][1] = D.m[i][j];
        Z.m[1][0] = D.m[j][i];
        Z.m[1][1] = D.m[j][j];
        mat r = mag_su2_max(&Z);
        if (bt)
            track_step2(bt, or_lipschitz(&r, omega, variant) * mag_max_amp(&Z), mag_rows(X, nc, i, j, 1),
                        mag_rows(X, nc, i, j, 0));
        r = overrelax(&r, omega, variant);
        mat R = mat_identity(nc);
        R.m[i][i] = r.m[0][0];
        R.m[i][j] = r.m[0][1];
        R.m[j][i] = r.m[1][0];
        R.m[j][j] = r.m[1][1];
        mat Rd = mat_adj(&R);
        for (int a = 0; a < nc; a++) {
            mat t = mat_mul(&R, &X[a]);
            X[a] = mat_mul(&t, &Rd);
        }
        g = mat_mul(&R, &g);
    }
    return g;
}

static mat mag_local_gauge(mat *X, int nc, double omega, int variant)
{
    return mag_local_gauge_b(X, nc, omega, variant, NULL);
}

/* The MAG site update; bc (or NULL) carries the error bounds: each X_a
 * starts with twice the gathered links' errors (U P U^+ moves by 2 ||dU||)
 * and is rotated on both sides by each subgroup step (nK = 2 x 8, F4). */
static void mag_update_site_b(double *U, const lattice *lat, int nc, long i, double omega, int variant,
                              const bound_ctx *bc)
{
    mat X[3];
    mag_X(U, lat, nc, i, X);
    bound_track bt;
    if (bc) bt = track_begin(bc, lat, i, 0, 2.0);
    double E0 = bc ? bt.E : 0.0;
    mat X0[3] = {X[0], X[1], X[2]};
    mat g = mag_local_gauge_b(X, nc, omega, variant, bc ? &bt : NULL);
    if (bc && bc->tight && nc == 3) {
        site_map m = {1, 0, omega, variant, 0.0, NULL, 0, 0};
        bt.dg = fmin(bt.dg, tangent_dg(&m, X0, E0, bc->rho));
    }
    mat gd = mat_adj(&g);
    for (int mu = 0; mu < 4; mu++) {
        long ib = site_shift(lat, i, mu, -1);
        mat f = get_link(U, nc, i, mu);
        mat b = get_link(U, nc, ib, mu);
        mat fn = mat_mul(&g, &f);
        mat bn = mat_mul(&b, &gd);
        put_link(U, nc, i, mu, &fn);
        put_link(U, nc, ib, mu, &bn);
    }
    if (bc) track_end(bc, &bt, lat, i, 0);
}

static void mag_update_site(double *U, const lattice *lat, int nc, long i, double omega, int variant)
{
    mag_update_site_b(U, lat, nc, i, omega, variant, NULL);
}

void oracle_mag_halfsweep(double *U, const int *L, int nc, int parity, double omega, int variant)
{
    lattice lat = make_lattice(L);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < lat.V; i++)
        if (site_parity(&lat, i, 0) == parity) mag_update_site(U, &lat, nc, i, omega, variant);
}

void oracle_mag_sweep(double *U, const int *L, int nc, double omega, int variant, int n_sweeps)
{
    for (int s = 0; s < n_sweeps; s++) {
        oracle_mag_halfsweep(U, L, nc, 0, omega, variant);
        oracle_mag_halfsweep(U, L, nc, 1, omega, variant);
    }
}

/* One MAG sweep, exactly as oracle_mag_sweep, with the error bounds of
 * oracle_sweep_bound. */
void oracle_mag_sweep_bound(double *U, const int *L, int nc, double omega, int variant, double rho, double *e,
                            int tight)
{
    lattice lat = make_lattice(L);
    bound_ctx bc = {e, NULL, rho, tight};
    for (int parity = 0; parity < 2; parity++) {
#pragma omp parallel for schedule(static)
        for (long i = 0; i < lat.V; i++)
            if (site_parity(&lat, i, 0) == parity) mag_update_site_b(U, &lat, nc, i, omega, variant, &bc);
    }
}

/* R15: the MAG condition is the stationarity of the local functional at
 * g = 1: its gradient sum_a [X_a, P_a] has the entries (X_j - X_i)_ij off the
 * diagonal (and 0 on it). theta_MAG = (1/V) sum_x sum_{i != j} |(X_i - X_j)_ij|^2;
 * F_MAG as in R12. Per-site values are summed in site order. */
void oracle_mag_theta(const double *U, const int *L, int nc, double *theta, double *F)
{
    lattice lat = make_lattice(L);
    double *th = (double *)malloc(sizeof(double) * lat.V);
    double *ff = (double *)malloc(sizeof(double) * lat.V);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < lat.V; i++) {
        mat X[3];
        mag_X(U, &lat, nc, i, X);
        double t = 0.0;
        for (int a = 0; a < nc; a++)
            for (int b = 0; b < nc; b++)
                if (a != b) t += c_abs2(c_sub(X[a].m[a][b], X[b].m[a][b]));
        th[i] = t;
        double f = 0.0;
        for (int mu = 0; mu < 4; mu++) {
            mat u = get_link(U, nc, i, mu);
            for (int a = 0; a < nc; a++) f += c_abs2(u.m[a][a]);
        }
        ff[i] = f;
    }
    double st = 0.0, sf = 0.0;
    for (long i = 0; i < lat.V; i++) {
        st += th[i];
        sf += ff[i];
    }
    free(th);
    free(ff);
    *theta = st / (double)lat.V;
    *F = sf / (4.0 * nc * (double)lat.V);
}

/* MAG fixing, with the stopping and reunitarisation rules of oracle_landau_fix. */
int oracle_mag_fix(double *U, const int *L, int nc, double omega, int variant, double theta_target, int max_sweeps,
                   int check_every, int reunit_every, int *sweeps_out, double *theta_out, double *F_out)
{
    lattice lat = make_lattice(L);
    double th, F;
    int n = 0;
    oracle_mag_theta(U, L, nc, &th, &F);
    while (!(th < theta_target) && n < max_sweeps) {
        for (int k = 0; k < check_every && n < max_sweeps; k++) {
            oracle_mag_sweep(U, L, nc, omega, variant, 1);
            n++;
            if (reunit_every > 0 && n % reunit_every == 0) oracle_reunitarize(U, lat.V * 4, nc);
        }
        oracle_mag_theta(U, L, nc, &th, &F);
    }
    *sweeps_out = n;
    *theta_out = th;
    *F_out = F;
    return th < theta_target ? 0 : 1;
}

/* the MAG site transformation for given X_0 .. X_{Nc-1} (Nc x Nc each); X is
 * rotated in place as the subgroup steps go */
void oracle_mag_local_gauge(double *X, int nc, double omega, int variant, double *g)
{
    mat Xm[3];
    for (int a = 0; a < nc; a++) Xm[a] = get_mat(X, nc, a);
    mat r = mag_local_gauge(Xm, nc, omega, variant);
    for (int a = 0; a < nc; a++) put_mat(X, nc, a, &Xm[a]);
    put_mat(g, nc, 0, &r);
}

/* The bound of mag_local_gauge_b: ||dg|| per unit of max_a ||dX_a||. */
double oracle_mag_local_gauge_bound(const double *X, int nc, double omega, int variant)
{
    mat Xm[3];
    for (int a = 0; a < nc; a++) Xm[a] = get_mat(X, nc, a);
    bound_track bt = {1.0, 0.0, 0.0, INFINITY};
    mag_local_gauge_b(Xm, nc, omega, variant, &bt);
    return bt.dg;
}

/* the SU(2) maximiser of (1/2) tr[s3 B Z B^+] for a 2x2 hermitian Z */
void oracle_mag_su2_max(const double *Z, double *B)
{
    mat z = get_mat(Z, 2, 0);
    mat b = mag_su2_max(&z);
    put_mat(B, 2, 0, &b);
}

/* R16: MAG heat bath. For the block vector z (R13) with n = |z| > 0 the
 * subgroup functional of B = C Bmax (Bmax the maximiser) is n (2u - 1) with
 * u = c0^2 + c3^2 for C = (c0, c1, c2, c3); under Haar measure u is uniform on
 * [0, 1], so the weight exp(functional / T) makes u exponential with rate
 * -beta, beta = 2 n / T, drawn by inversion: w = 1 - u = -log1p(v expm1(-beta)) / beta
 * and, for beta <= 30, u = log1p((1 - v) expm1(beta)) / beta (else 1 - w).
 * C = (sqrt(u) cos a, sqrt(w) cos c, sqrt(w) sin c, sqrt(u) sin a) with the
 * angles a = 2 pi v1, c = 2 pi v2 uniform. Counter (site, sweep, sub << 1, 0),
 * one Philox block per subgroup. n = 0 leaves the block alone. */
/* u and w = 1 - u of the draw of R16 for the uniform v0 */
static void mag_hb_uw(double beta, double v0, double *u, double *w)
{
    *w = -log1p(v0 * expm1(-beta)) / beta;
    *u = beta <= 30.0 ? log1p((1.0 - v0) * expm1(beta)) / beta : 1.0 - *w;
}

static mat mag_heatbath_su2(const mat *Z, double inv_T, const uint32_t *key, uint32_t site, uint32_t sweep, int sub,
                            bound_track *bt, double rows, double rows_rho)
{
    double z3 = 0.5 * (Z->m[0][0].re - Z->m[1][1].re);
    double z1 = Z->m[0][1].re, z2 = -Z->m[0][1].im;
    double n = sqrt(z1 * z1 + z2 * z2 + z3 * z3);
    if (!(n > 0.0)) {
        if (bt) track_step2(bt, INFINITY, rows, rows_rho);
        return mat_identity(2);
    }
    mat Bmax = mag_su2_max(Z);
    double beta = (2.0 * n) * inv_T;
    double v[4];
    draw4(key, site, sweep, (uint32_t)sub << 1, v);
    double u, w;
    mag_hb_uw(beta, v[0], &u, &w);
    if (bt) {
        /* B = C Bmax: Bmax moves by 2 E / N (mag_max_amp); beta = 2 |z| / T by
         * at most 4 E / T, and C with it by |dC/dbeta| per unit, C's
         * components being sqrt(u) and sqrt(w) times fixed unit vectors */
        double h = FD_STEP * beta, up, wp, um, wm;
        mag_hb_uw(beta + h, v[0], &up, &wp);
        mag_hb_uw(beta - h, v[0], &um, &wm);
        double a = (sqrt(fmax(up, 0.0)) - sqrt(fmax(um, 0.0))) / (2.0 * h);
        double b = (sqrt(fmax(wp, 0.0)) - sqrt(fmax(wm, 0.0))) / (2.0 * h);
        track_step2(bt, mag_max_amp(Z) + sqrt(a * a + b * b) * 4.0 * inv_T, rows, rows_rho);
    }
    double su = sqrt(u), sw = sqrt(w);
    double c[4] = {su * cos(TWO_PI * v[1]), sw * cos(TWO_PI * v[2]), sw * sin(TWO_PI * v[2]), su * sin(TWO_PI * v[1])};
    mat C = quaternion_matrix(c);
    mat B = mat_mul(&C, &Bmax);
    cplx s = c_sqrt(mat_det2(&B));
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) B.m[a][b] = c_div(B.m[a][b], s);
    return B;
}

/* the MAG heat-bath site transformation: the subgroups of R14 with the draw of
 * R16 in place of the overrelaxed maximiser */
static mat mag_heatbath_gauge(mat *X, int nc, double inv_T, const uint32_t *key, uint32_t site, uint32_t sweep,
                              bound_track *bt)
{
    static const int sub[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    int nsub = nc == 2 ? 1 : 3;
    mat g = mat_identity(nc);
    for (int s = 0; s < nsub; s++) {
        int i = sub[s][0], j = sub[s][1];
        mat D = mat_sub(&X[i], &X[j]);
        mat Z = mat_zero(2);
        Z.m[0][0] = D.m[i][i];
        Z.m[0][1] = D.m[i][j];
        Z.m[1][0] = D.m[j][i];
        Z.m[1][1] = D.m[j][j];
        mat r = mag_heatbath_su2(&Z, inv_T, key, site, sweep, s, bt, bt ? mag_rows(X, nc, i, j, 1) : 0.0,
                                 bt ? mag_rows(X, nc, i, j, 0) : 0.0);
        mat R = mat_identity(nc);
        R.m[i][i] = r.m[0][0];
        R.m[i][j] = r.m[0][1];
        R.m[j][i] = r.m[1][0];
        R.m[j][j] = r.m[1][1];
        mat Rd = mat_adj(&R);
        for (int a = 0; a < nc; a++) {
            mat t = mat_mul(&R, &X[a]);
            X[a] = mat_mul(&t, &Rd);
        }
        g = mat_mul(&R, &g);
    }
    return g;
}

static void mag_heatbath_site_b(double *U, const lattice *lat, int nc, long i, double inv_T, const uint32_t *key,
                                uint32_t sweep, const bound_ctx *bc)
{
    mat X[3];
    mag_X(U, lat, nc, i, X);
    bound_track bt;
    if (bc) bt = track_begin(bc, lat, i, 0, 2.0);
    double E0 = bc ? bt.E : 0.0;
    mat X0[3] = {X[0], X[1], X[2]};
    mat g = mag_heatbath_gauge(X, nc, inv_T, key, (uint32_t)i, sweep, bc ? &bt : NULL);
    if (bc && bc->tight && nc == 3) {
        site_map m = {1, 1, 0.0, 0, inv_T, key, (uint32_t)i, sweep};
        bt.dg = fmin(bt.dg, tangent_dg(&m, X0, E0, bc->rho));
    }
    mat gd = mat_adj(&g);
    for (int mu = 0; mu < 4; mu++) {
        long ib = site_shift(lat, i, mu, -1);
        mat f = get_link(U, nc, i, mu);
        mat b = get_link(U, nc, ib, mu);
        mat fn = mat_mul(&g, &f);
        mat bn = mat_mul(&b, &gd);
        put_link(U, nc, i, mu, &fn);
        put_link(U, nc, ib, mu, &bn);
    }
    if (bc) track_end(bc, &bt, lat, i, 0);
}

void oracle_mag_heatbath_halfsweep(double *U, const int *L, int nc, int parity, double T, const uint32_t *key,
                                   uint32_t sweep)
{
    lattice lat = make_lattice(L);
    double inv_T = 1.0 / T;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < lat.V; i++)
        if (site_parity(&lat, i, 0) == parity) mag_heatbath_site_b(U, &lat, nc, i, inv_T, key, sweep, NULL);
}

/* One MAG heat-bath sweep with the error bounds of oracle_sweep_bound (the
 * MAG draw takes no decisions, so there is no slack). */
void oracle_mag_heatbath_sweep_bound(double *U, const int *L, int nc, double T, const uint32_t *key, uint32_t sweep,
                                     double rho, double *e, int tight)
{
    lattice lat = make_lattice(L);
    bound_ctx bc = {e, NULL, rho, tight};
    double inv_T = 1.0 / T;
    for (int parity = 0; parity < 2; parity++) {
#pragma omp parallel for schedule(static)
        for (long i = 0; i < lat.V; i++)
            if (site_parity(&lat, i, 0) == parity) mag_heatbath_site_b(U, &lat, nc, i, inv_T, key, sweep, &bc);
    }
}

void oracle_mag_heatbath_sweep(double *U, const int *L, int nc, double T, const uint32_t *key, uint32_t sweep)
{
    oracle_mag_heatbath_halfsweep(U, L, nc, 0, T, key, sweep);
    oracle_mag_heatbath_halfsweep(U, L, nc, 1, T, key, sweep);
}

/* the schedule of R11 with MAG heat-bath sweeps and MAG microcanonical sweeps
 * (omega = 2: the smallest rotation applied twice keeps each block functional) */
void oracle_mag_anneal(double *U, const int *L, int nc, double t_start, double t_end, int steps, int n_micro,
                       const uint32_t *key, int reunit_every)
{
    lattice lat = make_lattice(L);
    long done = 0;
    for (int k = 0; k < steps; k++) {
        double T = steps > 1 ? t_start + (t_end - t_start) * (double)k / (double)(steps - 1) : t_start;
        for (int m = 0; m <= n_micro; m++) {
            if (m == 0)
                oracle_mag_heatbath_sweep(U, L, nc, T, key, (uint32_t)k);
            else
                oracle_mag_sweep(U, L, nc, 2.0, 0, 1);
            done++;
            if (reunit_every > 0 && done % reunit_every == 0) oracle_reunitarize(U, lat.V * 4, nc);
        }
    }
}

/* one MAG heat-bath subgroup draw for a 2x2 hermitian block Z */
void oracle_mag_heatbath_su2(const double *Z, double T, const uint32_t *key, uint32_t site, uint32_t sweep, int sub,
                             double *B)
{
    mat z = get_mat(Z, 2, 0);
    mat b = mag_heatbath_su2(&z, 1.0 / T, key, site, sweep, sub, NULL, 0.0, 0.0);
    put_mat(B, 2, 0, &b);
}

/* ------------------------------------------------------------------ */
/* single-matrix entry points for the pin tests                        */
/* ------------------------------------------------------------------ */

/* g for one gathered K (Nc x Nc complex, interleaved) */
void oracle_local_gauge(const double *K, int nc, double omega, int variant, double *g)
{
    mat k = get_mat(K, nc, 0);
    mat r = local_gauge(&k, omega, variant);
    put_mat(g, nc, 0, &r);
}

/* The bound of local_gauge_b for one K: ||dg|| per unit ||dK|| (no rounding
 * charges), i.e. the site's amplification of an error in its gathered K. */
double oracle_local_gauge_bound(const double *K, int nc, double omega, int variant)
{
    mat k = get_mat(K, nc, 0);
    bound_track bt = {1.0, 0.0, 0.0, INFINITY};
    local_gauge_b(&k, omega, variant, &bt);
    return bt.dg;
}

/* the SU(2) maximiser of Re tr[r w] for a 2x2 block w (no overrelaxation) */
void oracle_su2_local_max(const double *w, double *r)
{
    mat a = get_mat(w, 2, 0);
    mat b = su2_local_max(&a);
    put_mat(r, 2, 0, &b);
}

/* the heat-bath transformation of one site for a gathered K at temperature T,
 * drawn with counter words (site, sweep) */
void oracle_heatbath_gauge(const double *K, int nc, double T, const uint32_t *key, uint32_t site, uint32_t sweep,
                           double *g)
{
    mat k = get_mat(K, nc, 0);
    mat r = heatbath_gauge(&k, 1.0 / T, key, site, sweep, NULL);
    put_mat(g, nc, 0, &r);
}

/* The bound of the heat-bath site transformation for one K: ||dg|| per unit
 * ||dK|| with the draws' decisions held (no rounding charges); *slack
 * receives the smallest decision slack for errors of K up to dK. */
double oracle_heatbath_gauge_bound(const double *K, int nc, double T, const uint32_t *key, uint32_t site,
                                   uint32_t sweep, double dK, double *slack)
{
    mat k = get_mat(K, nc, 0);
    bound_track bt = {dK, 0.0, 0.0, INFINITY};
    heatbath_gauge(&k, 1.0 / T, key, site, sweep, &bt);
    if (slack) *slack = bt.slack;
    return bt.dg / dK;
}

/* g^omega for one SU(2) matrix */
void oracle_overrelax(const double *g, double omega, int variant, double *out)
{
    mat a = get_mat(g, 2, 0);
    mat b = overrelax(&a, omega, variant);
    put_mat(out, 2, 0, &b);
}

/* ------------------------------------------------------------------ */
/* tight first-order bounds of an SU(3) site: its tangent map          */
/* ------------------------------------------------------------------ */
/* F1-F5 bound each subgroup step by norms and compound the bounds over the
 * three steps of an SU(3) site, which overstates the first-order response
 * of g by tens (hundreds and more on the random start). tangent_dg carries
 * the site's first-order map itself: every unit direction of its input (the
 * 18 real components of K, or a hermitian basis of each X_a) goes through
 * the exact derivative of each step (the block maximiser, the
 * overrelaxation or the draw, the rotation of the running matrix, the
 * product into g), and the bound is the operator norm of the resulting
 * linear map onto the tangent space of g. Rounding is charged as in F1-F5,
 * sqrt2 rho on g per step and rho times the rotated rows (F3; MAG: twice
 * the rows of X_a) on the running matrix, each charge carried by the exact
 * map of the steps after it. For the heat bath this covers errors of the
 * input, not the draw's own rounding, which can move x by thousands of
 * units where a small cosine multiplies log u2 (R10): comparisons of heat-
 * bath sweeps with another implementation take the norm bound. It bounds the same first-order quantity as the
 * norm rules, so the smaller of the two holds. */

static const int SUB3[3][2] = {{0, 1}, {0, 2}, {1, 2}};

/* d/dt det(A + t dA) at t = 0 for 2x2 matrices (real part: real for the
 * quaternion-type pairs here) */
static double det2_dir(const mat *A, const mat *dA)
{
    cplx t = c_add(c_mul(A->m[1][1], dA->m[0][0]), c_mul(A->m[0][0], dA->m[1][1]));
    t = c_sub(t, c_add(c_mul(A->m[0][1], dA->m[1][0]), c_mul(A->m[1][0], dA->m[0][1])));
    return t.re;
}

/* (A - B s) / n for 2x2 matrices */
static mat comb2(const mat *A, const mat *B, double s, double n)
{
    mat out = mat_zero(2);
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) out.m[a][b] = c_scale(c_sub(A->m[a][b], c_scale(B->m[a][b], s)), 1.0 / n);
    return out;
}

/* derivative of su2_local_max at w along dw, for det P(w) > 0:
 * r = q^+ / n with q = P(w), n = sqrt(det q), so dr = (dq^+ - r dn) / n */
static mat su2_max_dir(const mat *w, const mat *dw)
{
    mat q = su2_part(w), dq = su2_part(dw);
    double n = sqrt(fmax(mat_det2(&q).re, 0.0));
    double dn = 0.5 * det2_dir(&q, &dq) / n;
    mat qd = mat_adj(&q), dqd = mat_adj(&dq);
    return comb2(&dqd, &qd, dn / n, n);
}

/* derivative of mag_su2_max at Z along dZ, for |z| > 0 and z off -e3:
 * B = M / s with s = sqrt(det M), so dB = (dM - B ds) / s */
static mat mag_max_dir(const mat *Z, const mat *dZ)
{
    double z3 = 0.5 * (Z->m[0][0].re - Z->m[1][1].re), z1 = Z->m[0][1].re, z2 = -Z->m[0][1].im;
    double d3 = 0.5 * (dZ->m[0][0].re - dZ->m[1][1].re), d1 = dZ->m[0][1].re, d2 = -dZ->m[0][1].im;
    double n = sqrt(z1 * z1 + z2 * z2 + z3 * z3);
    double dn = (z1 * d1 + z2 * d2 + z3 * d3) / n;
    mat M = mat_zero(2), dM = mat_zero(2);
    M.m[0][0] = M.m[1][1] = c_make(n + z3, 0.0);
    M.m[0][1] = c_make(z1, -z2);
    M.m[1][0] = c_make(-z1, -z2);
    dM.m[0][0] = dM.m[1][1] = c_make(dn + d3, 0.0);
    dM.m[0][1] = c_make(d1, -d2);
    dM.m[1][0] = c_make(-d1, -d2);
    double s = sqrt(mat_det2(&M).re);
    double ds = 0.5 * det2_dir(&M, &dM) / s;
    return comb2(&dM, &M, ds / s, s);
}

/* derivative of overrelax at the SU(2) element r along the tangent dr;
 * *ok = 0 where the map has none (variant 1 at r = -1) */
static mat or_dir(const mat *r, const mat *dr, double omega, int variant, int *ok)
{
    mat out = mat_zero(2);
    if (variant == 0) {
        /* G = 1 + omega D + c D^2 (D = r - 1), out = G / sqrt(det G) */
        double c = 0.5 * omega * (omega - 1.0);
        mat one = mat_identity(2);
        mat D = mat_sub(r, &one);
        mat D2 = mat_mul(&D, &D);
        mat t1 = mat_scale(&D, c_make(omega, 0.0)), t2 = mat_scale(&D2, c_make(c, 0.0));
        mat G = mat_add(&one, &t1);
        G = mat_add(&G, &t2);
        mat a1 = mat_mul(dr, &D), a2 = mat_mul(&D, dr);
        mat dG = mat_add(&a1, &a2);
        dG = mat_scale(&dG, c_make(c, 0.0));
        mat o1 = mat_scale(dr, c_make(omega, 0.0));
        dG = mat_add(&dG, &o1);
        double m = sqrt(fmax(mat_det2(&G).re, 0.0));
        if (!(m > 0.0)) {
            *ok = 0;
            return out;
        }
        double dm = 0.5 * det2_dir(&G, &dG) / m;
        mat Gm = mat_scale(&G, c_make(1.0 / m, 0.0));
        return comb2(&dG, &Gm, dm, m);
    }
    /* out = cos(omega phi) 1 + f S, S = (r - r^+)/2, f = sin(omega phi) / sin(phi) */
    mat rd = mat_adj(r);
    mat S = mat_sub(r, &rd);
    S = mat_scale(&S, c_make(0.5, 0.0));
    double cphi = 0.5 * mat_trace(r).re;
    double sphi = sqrt(fmax(mat_det2(&S).re, 0.0));
    if (sphi == 0.0) {
        if (cphi > 0.0) return mat_scale(dr, c_make(omega, 0.0)); /* r^omega at r = 1 */
        *ok = 0;
        return out;
    }
    double phi = atan2(sphi, cphi);
    mat drd = mat_adj(dr);
    mat dS = mat_sub(dr, &drd);
    dS = mat_scale(&dS, c_make(0.5, 0.0));
    double dc = 0.5 * mat_trace(dr).re;
    double ds = 0.5 * det2_dir(&S, &dS) / sphi;
    double dphi = (cphi * ds - sphi * dc) / (cphi * cphi + sphi * sphi);
    double f = sin(omega * phi) / sphi;
    double df = (omega * cos(omega * phi) * dphi - f * ds) / sphi;
    mat p1 = mat_scale(&dS, c_make(f, 0.0)), p2 = mat_scale(&S, c_make(df, 0.0));
    out = mat_add(&p1, &p2);
    double dd = -omega * sin(omega * phi) * dphi;
    out.m[0][0] = c_add(out.m[0][0], c_make(dd, 0.0));
    out.m[1][1] = c_add(out.m[1][1], c_make(dd, 0.0));
    return out;
}

/* One subgroup step, linearised: the block, the maximiser v (Landau) or
 * Bmax (MAG), the SU(2) element applied, and for the heat bath the drawn
 * quaternion X with its derivative per unit alpha (beta) at the same
 * uniforms, a central difference as in hb_track */
typedef struct {
    mat blk, v, r, X;
    double xp[4];
    double k; /* Landau: sqrt(det P(w)); MAG: |z| */
    int ok;
} step_lin;

/* the 2x2 block of step s: of K (Landau), or of X_i - X_j (MAG) */
static mat block_of(const site_map *m, const mat *S, int s)
{
    int i = SUB3[s][0], j = SUB3[s][1];
    mat D = m->mag ? mat_sub(&S[i], &S[j]) : S[0];
    mat w = mat_zero(2);
    w.m[0][0] = D.m[i][i];
    w.m[0][1] = D.m[i][j];
    w.m[1][0] = D.m[j][i];
    w.m[1][1] = D.m[j][j];
    return w;
}

static void lin_step(const site_map *m, const mat *blk, int s, step_lin *L)
{
    L->blk = *blk;
    L->ok = 1;
    if (!m->mag) {
        mat q = su2_part(blk);
        L->k = sqrt(fmax(mat_det2(&q).re, 0.0));
        if (!(L->k > 0.0)) {
            L->ok = 0;
            return;
        }
        L->v = su2_local_max(blk);
        if (!m->hb) {
            L->r = overrelax(&L->v, m->omega, m->variant);
            return;
        }
        L->r = heatbath_su2(blk, m->inv_T, m->key, m->site, m->sweep, s, NULL, 0.0);
        double alpha = (2.0 * L->k) * m->inv_T, h = FD_STEP * alpha, x[4], xa[4], xb[4];
        oracle_hb_x(alpha, m->key, m->site, m->sweep, s, x);
        oracle_hb_x(alpha + h, m->key, m->site, m->sweep, s, xa);
        oracle_hb_x(alpha - h, m->key, m->site, m->sweep, s, xb);
        for (int c = 0; c < 4; c++) L->xp[c] = (xa[c] - xb[c]) / (2.0 * h);
        L->X = quaternion_matrix(x);
        return;
    }
    double z3 = 0.5 * (blk->m[0][0].re - blk->m[1][1].re), z1 = blk->m[0][1].re, z2 = -blk->m[0][1].im;
    L->k = sqrt(z1 * z1 + z2 * z2 + z3 * z3);
    if (!(L->k > 0.0) || !(L->k + z3 > 0.0)) {
        L->ok = 0;
        return;
    }
    L->v = mag_su2_max(blk);
    if (!m->hb) {
        L->r = overrelax(&L->v, m->omega, m->variant);
        return;
    }
    L->r = mag_heatbath_su2(blk, m->inv_T, m->key, m->site, m->sweep, s, NULL, 0.0, 0.0);
    double beta = (2.0 * L->k) * m->inv_T, h = FD_STEP * beta, v[4], u, w, up, wp, um, wm;
    draw4(m->key, m->site, m->sweep, (uint32_t)s << 1, v);
    mag_hb_uw(beta, v[0], &u, &w);
    mag_hb_uw(beta + h, v[0], &up, &wp);
    mag_hb_uw(beta - h, v[0], &um, &wm);
    double a = (sqrt(fmax(up, 0.0)) - sqrt(fmax(um, 0.0))) / (2.0 * h);
    double b = (sqrt(fmax(wp, 0.0)) - sqrt(fmax(wm, 0.0))) / (2.0 * h);
    double ca = cos(TWO_PI * v[1]), sa = sin(TWO_PI * v[1]), cc = cos(TWO_PI * v[2]), sc = sin(TWO_PI * v[2]);
    double c[4] = {sqrt(u) * ca, sqrt(w) * cc, sqrt(w) * sc, sqrt(u) * sa};
    L->X = quaternion_matrix(c);
    L->xp[0] = a * ca;
    L->xp[1] = b * cc;
    L->xp[2] = b * sc;
    L->xp[3] = a * sa;
}

/* the step's SU(2) element moved along the block's tangent dblk */
static mat step_dr(const site_map *m, const step_lin *L, const mat *dblk, int *ok)
{
    mat dv = m->mag ? mag_max_dir(&L->blk, dblk) : su2_max_dir(&L->blk, dblk);
    if (!m->hb) return or_dir(&L->v, &dv, m->omega, m->variant, ok);
    /* heat bath: r = X v, X moving with alpha = 2 k / T (MAG: beta = 2 |z| / T) */
    double dk;
    if (!m->mag) {
        mat q = su2_part(&L->blk), dq = su2_part(dblk);
        dk = 0.5 * det2_dir(&q, &dq) / L->k;
    } else {
        double z3 = 0.5 * (L->blk.m[0][0].re - L->blk.m[1][1].re), z1 = L->blk.m[0][1].re,
               z2 = -L->blk.m[0][1].im;
        double d3 = 0.5 * (dblk->m[0][0].re - dblk->m[1][1].re), d1 = dblk->m[0][1].re, d2 = -dblk->m[0][1].im;
        dk = (z1 * d1 + z2 * d2 + z3 * d3) / L->k;
    }
    double dpar = 2.0 * dk * m->inv_T, dx[4];
    for (int c = 0; c < 4; c++) dx[c] = L->xp[c] * dpar;
    mat dX = quaternion_matrix(dx);
    mat t1 = mat_mul(&dX, &L->v), t2 = mat_mul(&L->X, &dv);
    return mat_add(&t1, &t2);
}

/* 3x3 with the 2x2 block b at rows/columns i, j; `one` = 1 elsewhere on the diagonal, else 0 */
static mat embed3(const mat *b, int i, int j, int one)
{
    mat R = one ? mat_identity(3) : mat_zero(3);
    R.m[i][i] = b->m[0][0];
    R.m[i][j] = b->m[0][1];
    R.m[j][i] = b->m[1][0];
    R.m[j][j] = b->m[1][1];
    return R;
}

/* coordinates of an element of su(3) (anti-hermitian, traceless) in an
 * orthonormal basis: sqrt2 Re, Im of the entries above the diagonal and two
 * combinations of the diagonal's imaginary parts; their Euclidean norm is
 * the Frobenius norm */
static void su3_coords(const mat *X, double *c)
{
    c[0] = SQRT2 * X->m[0][1].re;
    c[1] = SQRT2 * X->m[0][1].im;
    c[2] = SQRT2 * X->m[0][2].re;
    c[3] = SQRT2 * X->m[0][2].im;
    c[4] = SQRT2 * X->m[1][2].re;
    c[5] = SQRT2 * X->m[1][2].im;
    c[6] = (X->m[0][0].im - X->m[1][1].im) / SQRT2;
    c[7] = (X->m[0][0].im + X->m[1][1].im - 2.0 * X->m[2][2].im) / sqrt(6.0);
}

/* ||J||_2 from above for the 8 x n matrix J (column c at J + 8 c): for the
 * symmetric M = J J^T >= 0, lambda_max^16 <= tr M^16 <= 8 lambda_max^16, so
 * (tr M^16)^(1/32) is at most 8^(1/32) = 1.067 times ||J||_2. M^16 by four
 * squarings, each renormalised to unit trace, the traces kept as logs. */
static double opnorm8(const double *J, int n)
{
    double M[8][8], T[8][8];
    for (int a = 0; a < 8; a++)
        for (int b = 0; b < 8; b++) {
            double s = 0.0;
            for (int c = 0; c < n; c++) s += J[8 * c + a] * J[8 * c + b];
            M[a][b] = s;
        }
    double t = 0.0;
    for (int a = 0; a < 8; a++) t += M[a][a];
    if (!(t > 0.0)) return t == 0.0 ? 0.0 : INFINITY;
    double lg = 16.0 * log(t), p = 8.0;
    for (int a = 0; a < 8; a++)
        for (int b = 0; b < 8; b++) M[a][b] /= t;
    for (int k = 0; k < 4; k++) {
        t = 0.0;
        for (int a = 0; a < 8; a++)
            for (int b = 0; b < 8; b++) {
                double s = 0.0;
                for (int c = 0; c < 8; c++) s += M[a][c] * M[c][b];
                T[a][b] = s;
            }
        for (int a = 0; a < 8; a++) t += T[a][a];
        for (int a = 0; a < 8; a++)
            for (int b = 0; b < 8; b++) M[a][b] = T[a][b] / t;
        lg += p * log(t);
        p *= 0.5;
    }
    return exp(lg / 32.0);
}

/* unit direction d of the site's input: K (18 real components), or the
 * hermitian basis of each X_a (9 per a: diagonal units, then the symmetric
 * and antisymmetric pairs of each entry above the diagonal over sqrt2) */
static void unit_dir(const site_map *m, int d, mat *dS)
{
    for (int a = 0; a < 3; a++) dS[a] = mat_zero(3);
    if (!m->mag) {
        int e = d / 2;
        dS[0].m[e / 3][e % 3] = (d & 1) ? c_make(0.0, 1.0) : c_make(1.0, 0.0);
        return;
    }
    int a = d / 9, e = d % 9;
    if (e < 3) {
        dS[a].m[e][e] = c_make(1.0, 0.0);
        return;
    }
    static const int pr[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    int k = pr[(e - 3) / 2][0], l = pr[(e - 3) / 2][1];
    if ((e - 3) % 2 == 0) {
        dS[a].m[k][l] = c_make(1.0 / SQRT2, 0.0);
        dS[a].m[l][k] = c_make(1.0 / SQRT2, 0.0);
    } else {
        dS[a].m[k][l] = c_make(0.0, 1.0 / SQRT2);
        dS[a].m[l][k] = c_make(0.0, -1.0 / SQRT2);
    }
}

/* Operator norm (from above) of the map from the running input at step s0
 * to the tangent of g through steps s0..2: Landau ||J||, MAG the sum over a
 * of ||J_a|| (per unit max_a ||dX_a||). S[s] are the running inputs, L[s]
 * the steps, R[s] their 3x3 rotations. */
static double tail_norm(const site_map *m, mat S[4][3], const step_lin *L, const mat *R, int s0)
{
    if (s0 == 3) return 0.0;
    int nin = m->mag ? 27 : 18;
    double J[27 * 8];
    for (int d = 0; d < nin; d++) {
        mat dS[3];
        unit_dir(m, d, dS);
        mat dg = mat_zero(3), gt = mat_identity(3);
        for (int s = s0; s < 3; s++) {
            int i = SUB3[s][0], j = SUB3[s][1], ok = 1;
            mat dblk = block_of(m, dS, s);
            mat dr = step_dr(m, &L[s], &dblk, &ok);
            if (!ok) return INFINITY;
            mat dR = embed3(&dr, i, j, 0);
            if (!m->mag) {
                mat t1 = mat_mul(&dR, &S[s][0]), t2 = mat_mul(&R[s], &dS[0]);
                dS[0] = mat_add(&t1, &t2);
            } else {
                /* X_a' = R X_a R^+: dX_a' = Y + Y^+ + R dX_a R^+, Y = dR X_a R^+ */
                mat Rd = mat_adj(&R[s]);
                for (int a = 0; a < 3; a++) {
                    mat P = mat_mul(&S[s][a], &Rd);
                    mat Y = mat_mul(&dR, &P);
                    mat Yd = mat_adj(&Y);
                    mat t = mat_mul(&R[s], &dS[a]);
                    mat Q = mat_mul(&t, &Rd);
                    dS[a] = mat_add(&Y, &Yd);
                    dS[a] = mat_add(&dS[a], &Q);
                }
            }
            mat t1 = mat_mul(&dR, &gt), t2 = mat_mul(&R[s], &dg);
            dg = mat_add(&t1, &t2);
            gt = mat_mul(&R[s], &gt);
        }
        mat gtd = mat_adj(&gt);
        mat X = mat_mul(&dg, &gtd);
        su3_coords(&X, J + 8 * d);
    }
    if (!m->mag) return opnorm8(J, 18);
    return opnorm8(J, 9) + opnorm8(J + 72, 9) + opnorm8(J + 144, 9);
}

/* The tangent bound on ||dg|| of an SU(3) site whose input (K, or the X_a)
 * is known to within E, with rho per rounding step. */
static double tangent_dg(const site_map *m, const mat *state, double E, double rho)
{
    mat S[4][3];
    step_lin L[3];
    mat R[3];
    double rr[3], amp[4];
    int ns = m->mag ? 3 : 1;
    for (int a = 0; a < ns; a++) S[0][a] = state[a];
    for (int s = 0; s < 3; s++) {
        int i = SUB3[s][0], j = SUB3[s][1];
        mat blk = block_of(m, S[s], s);
        lin_step(m, &blk, s, &L[s]);
        if (!L[s].ok) return INFINITY;
        R[s] = embed3(&L[s].r, i, j, 1);
        rr[s] = m->mag ? mag_rows(S[s], 3, i, j, 0) : rows_norm(&S[s][0], i, j);
        if (!m->mag) {
            S[s + 1][0] = mat_mul(&R[s], &S[s][0]);
        } else {
            mat Rd = mat_adj(&R[s]);
            for (int a = 0; a < 3; a++) {
                mat t = mat_mul(&R[s], &S[s][a]);
                S[s + 1][a] = mat_mul(&t, &Rd);
            }
        }
    }
    for (int s0 = 0; s0 <= 3; s0++) amp[s0] = tail_norm(m, S, L, R, s0);
    double dg = amp[0] * E;
    for (int s = 0; s < 3; s++) dg += SQRT2 * rho + amp[s + 1] * rr[s] * rho;
    return dg;
}

/* The tangent bound of one SU(3) site map with no rounding: ||dg|| per unit
 * ||dK|| (mag = 0; in = K) or per unit max_a ||dX_a|| (mag = 1; in = X_0..2),
 * for overrelaxation (hb = 0) or the heat bath at T (hb = 1, draws of
 * (key, site, sweep)). */
double oracle_tangent_bound(const double *in, int mag, int hb, double omega, int variant, double T,
                            const uint32_t *key, uint32_t site, uint32_t sweep)
{
    mat S[3];
    for (int a = 0; a < (mag ? 3 : 1); a++) S[a] = get_mat(in, 3, a);
    site_map m = {mag, hb, omega, variant, hb ? 1.0 / T : 0.0, key, site, sweep};
    return tangent_dg(&m, S, 1.0, 0.0);
}

/* The MAG heat-bath site transformation of the X_a (consumed) into g. */
void oracle_mag_heatbath_gauge(double *X, int nc, double T, const uint32_t *key, uint32_t site, uint32_t sweep,
                               double *g)
{
    mat Xm[3];
    for (int a = 0; a < nc; a++) Xm[a] = get_mat(X, nc, a);
    mat G = mag_heatbath_gauge(Xm, nc, 1.0 / T, key, site, sweep, NULL);
    put_mat(g, nc, 0, &G);
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
