/*
 * Plain CPU oracle of the per-time-step test-particle update of CuBA
 * (Cardoso, Bicudo, Eilhauer, Bouras, "CuBA - a CUDA implementation of BAMPS",
 * arXiv:1208.0961): free streaming (Eq. 2), elastic reflection at the six box
 * walls (Sec. 2), binning into cells (Sec. 2, particles-in-a-cell method), and
 * binary 2->2 collisions inside a cell with probability
 * P22 = v_rel * sigma / N_test * dt / V_cell (Eq. 3), v_rel = s / (2 E1 E2),
 * followed by an isotropic re-direction in the centre-of-mass frame (Sec. 2).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  It shares nothing with the
 * CUDA library: its Philox generator, its sort, its arithmetic are written
 * here again, one particle and one pair at a time, in the order the method
 * states.  It is slow on purpose.
 *
 * Precision: FP64 throughout.  With params.fp32 = 1 the streaming, the cell
 * key and the P22 test are evaluated in IEEE single precision instead (a mirror
 * of a single-precision state), so that an FP32 implementation can be compared
 * with identical float arithmetic.  Kinematics and observables stay FP64.
 * Compile with -ffp-contract=off so that no multiply-add is fused.
 *
 * Readings where the paper is silent (each repeated at its function):
 *  - step order: stream -> reflect -> key -> stable sort -> pair test ->
 *    conflicts -> kinematics (the paper's flowchart figure is lost);
 *  - random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the seed,
 *    counters (step, cell, i, tag|j) as documented at each use;
 *  - conflicts: accepted pairs of a cell are executed greedily in
 *    lexicographic (i, j) order; a pair whose particle already collided in
 *    this step is dropped;
 *  - v_rel of massless particles is written 1/2 |n_i - n_j|^2 (= 1 - cos theta
 *    = s / (2 E_i E_j)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_INVALID (-1)
#define ORC_ERR_OOM (-2)

typedef struct {
    double L[3];      /* box edge lengths, fm */
    int32_t n[3];     /* cells per axis */
    double dt;        /* time step, fm/c */
    double sigma;     /* total isotropic cross section, fm^2 */
    double n_test;    /* test particles per physical particle */
    int32_t fp32;     /* 1: single-precision mirror of stream, key and P22 */
    uint32_t key[2];  /* Philox key (seed low word, seed high word) */
    int32_t skip;     /* 0: every pair tested (Eq. 3); 1: skip-ahead candidates + thinning */
    double kappa;     /* > 0: adaptive time step, dt is its upper bound (see orc_adaptive_dt) */
    double mass;      /* particle mass, GeV (0: massless gluons) */
    double mu;        /* > 0: screened forward-peaked angular distribution (see kin_general) */
} orc_params;

typedef struct {
    double lo[3], hi[3]; /* axis-aligned box, fm */
    double T;            /* temperature, GeV */
} orc_region;

typedef struct {
    uint32_t *keys;      /* [n] cell key after streaming, pre-sort order (or NULL) */
    int64_t *perm;       /* [n] sorted position -> pre-sort index (or NULL) */
    int64_t *cell_start; /* [ncells + 1] (or NULL) */
    uint32_t *acc;       /* [3 * acc_cap] accepted (cell, i, j), lexicographic (or NULL) */
    int64_t acc_cap, n_acc;
    uint32_t *exe;       /* [3 * exe_cap] executed (cell, i, j), lexicographic (or NULL) */
    int64_t exe_cap, n_exe;
    int64_t n_reflections;
    int64_t n_pairs_tested;
    int64_t n_candidates;  /* skip-ahead: candidate pairs drawn (P22 evaluated) */
    double dt;             /* the step's time step */
} orc_trace;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from Salmon, Moraes, Dror & Shaw, "Parallel random numbers: */
/* as easy as 1, 2, 3", SC'11: ten rounds of two 32x32->64 multiplications   */
/* with a Weyl-sequence key schedule.                                         */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox(uint32_t a, uint32_t b, uint32_t c, uint32_t d, const uint32_t key[2], uint32_t out[4])
{
    uint32_t ctr[4] = {a, b, c, d};
    orc_philox4x32_10(ctr, key, out);
}

/* Counter tags of the random streams (fourth counter word).                 */
#define TAG_MID 0x20000000u    /* acceptance: bits 23..16 of u_ij           */
#define TAG_FINE 0x40000000u   /* acceptance: low 16 bits of u_ij           */
#define TAG_ANGLE 0x80000000u  /* kinematics: CM-frame direction           */
#define TAG_SKIP 0xC0000000u   /* skip-ahead: k-th candidate draw of a row   */
#define TAG_MASS 0x40000000u   /* sampling of a massive momentum: try k      */
#define STEP_INIT 0xFFFFFFFFu  /* first counter word reserved for sampling */

/* ------------------------------------------------------------------------ */
/* Derived constants                                                         */
/* ------------------------------------------------------------------------ */
static double cell_len(const orc_params *p, int a) { return p->L[a] / (double)p->n[a]; }

static double cell_volume(const orc_params *p)
{
    /* V_cell = dx dy dz (Sec. 2). */
    return (cell_len(p, 0) * cell_len(p, 1)) * cell_len(p, 2);
}

/* C = sigma dt / (N_test V_cell): P22 = C v_rel (Eq. 3). */
double orc_p22_scale(const orc_params *p)
{
    return (p->sigma * p->dt) / (p->n_test * cell_volume(p));
}

int64_t orc_ncells(const orc_params *p) { return (int64_t)p->n[0] * p->n[1] * p->n[2]; }

static int check_params(const orc_params *p)
{
    for (int a = 0; a < 3; ++a) {
        if (!(p->L[a] > 0.0) || p->n[a] < 1) return ORC_ERR_INVALID;
        /* Results section: dt is chosen below the cell size, so a particle
           crosses at most one cell face per axis in a step. */
        if (!(p->dt < cell_len(p, a))) return ORC_ERR_INVALID;
    }
    if (!(p->dt > 0.0) || !(p->sigma >= 0.0) || !(p->n_test > 0.0)) return ORC_ERR_INVALID;
    if (p->skip != 0 && p->skip != 1) return ORC_ERR_INVALID;
    if (!(p->kappa >= 0.0) || p->kappa > 0.5) return ORC_ERR_INVALID;
    if (!(p->mass >= 0.0) || !(p->mu >= 0.0)) return ORC_ERR_INVALID;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Initial state: thermal Boltzmann gas of massless particles in boxes       */
/* ------------------------------------------------------------------------ */

/* Uniform variate in the open interval (0, 1) from a 32-bit word. */
static double open01(uint32_t r) { return ((double)r + 0.5) * 0x1p-32; }

/*
 * Momentum magnitude of a thermal particle at temperature T.  Massless: the
 * given Gamma(3, T) variate p0 (E = |p|, density p^2 exp(-p/T)).  Massive
 * (mass m > 0), the Juttner density p^2 exp(-sqrt(p^2 + m^2)/T) by rejection
 * from the massless one: try k draws the block (STEP_INIT, g_lo, g_hi,
 * TAG_MASS | k), proposes q = -T ln(u0 u1 u2) and keeps it iff
 * u3 < exp(-(sqrt(q^2 + m^2) - q) / T) (the ratio of the two densities, at
 * most 1; the difference written m^2 / (sqrt(q^2 + m^2) + q)).  After 64
 * rejected tries the last proposal is kept.
 */
static double sample_pmag(const orc_params *p, double T, uint32_t glo, uint32_t ghi, double p0)
{
    if (!(p->mass > 0.0)) return p0;
    const double m2 = p->mass * p->mass;
    double q = p0;
    for (uint32_t k = 0; k < 64; ++k) {
        uint32_t w[4];
        philox(STEP_INIT, glo, ghi, TAG_MASS | k, p->key, w);
        q = -T * log(open01(w[0]) * open01(w[1]) * open01(w[2]));
        double acc = exp(-(m2 / (sqrt(q * q + m2) + q)) / T);
        if (open01(w[3]) < acc) break;
    }
    return q;
}

/*
 * Number of particles per region: proportional to T^3 V (a Boltzmann gas has
 * n ∝ T^3), rounded by largest remainder (ties to the lower region index).
 */
int orc_region_counts(int64_t n, const orc_region *R, int nreg, int64_t *counts)
{
    if (nreg < 1 || n < 0) return ORC_ERR_INVALID;
    double wsum = 0.0;
    double *w = (double *)malloc(sizeof(double) * (size_t)nreg);
    if (!w) return ORC_ERR_OOM;
    for (int r = 0; r < nreg; ++r) {
        double v = 1.0;
        for (int a = 0; a < 3; ++a) v *= (R[r].hi[a] - R[r].lo[a]);
        if (!(v > 0.0) || !(R[r].T > 0.0)) { free(w); return ORC_ERR_INVALID; }
        w[r] = R[r].T * R[r].T * R[r].T * v;
        wsum += w[r];
    }
    int64_t assigned = 0;
    double *frac = (double *)malloc(sizeof(double) * (size_t)nreg);
    if (!frac) { free(w); return ORC_ERR_OOM; }
    for (int r = 0; r < nreg; ++r) {
        double q = (double)n * w[r] / wsum;
        counts[r] = (int64_t)floor(q);
        frac[r] = q - (double)counts[r];
        assigned += counts[r];
    }
    while (assigned < n) {
        int best = 0;
        for (int r = 1; r < nreg; ++r)
            if (frac[r] > frac[best]) best = r;
        counts[best] += 1;
        frac[best] = -1.0;
        assigned += 1;
    }
    free(w);
    free(frac);
    return ORC_OK;
}

/*
 * Sample n particles, region by region, in generation order.  Particle g uses
 * two Philox blocks with counters (STEP_INIT, g_lo, g_hi, 0) and (…, 1):
 * words a0..a2 place it uniformly in its region, E = -T ln(u1 u2 u3) with
 * (a3, b0, b1) samples the massless Boltzmann spectrum E^2 exp(-E/T)
 * (a Gamma(3, T) variate; massive particles: sample_pmag), and (b2, b3) give
 * an isotropic direction.
 * State layout: st[0..n) = x, [n..2n) = y, [2n..3n) = z, then px, py, pz.
 */
int orc_init_thermal(const orc_params *p, int64_t n, const orc_region *R, int nreg, double *st)
{
    if (check_params(p) != ORC_OK) return ORC_ERR_INVALID;
    int64_t *counts = (int64_t *)malloc(sizeof(int64_t) * (size_t)nreg);
    if (!counts) return ORC_ERR_OOM;
    int rc = orc_region_counts(n, R, nreg, counts);
    if (rc != ORC_OK) { free(counts); return rc; }
    int64_t g0 = 0;
    for (int r = 0; r < nreg; ++r) {
        const orc_region *reg = &R[r];
        for (int64_t k = 0; k < counts[r]; ++k) {
            int64_t g = g0 + k;
            uint32_t a[4], b[4];
            philox(STEP_INIT, (uint32_t)g, (uint32_t)((uint64_t)g >> 32), 0u, p->key, a);
            philox(STEP_INIT, (uint32_t)g, (uint32_t)((uint64_t)g >> 32), 1u, p->key, b);
            double pos[3];
            for (int ax = 0; ax < 3; ++ax)
                pos[ax] = reg->lo[ax] + open01(a[ax]) * (reg->hi[ax] - reg->lo[ax]);
            double E = sample_pmag(p, reg->T, (uint32_t)g, (uint32_t)((uint64_t)g >> 32),
                                   -reg->T * log(open01(a[3]) * open01(b[0]) * open01(b[1])));
            double ct = 2.0 * open01(b[2]) - 1.0;
            double stt = sqrt((1.0 - ct) * (1.0 + ct));
            double phi = 2.0 * M_PI * open01(b[3]);
            double mom[3] = {E * stt * cos(phi), E * stt * sin(phi), E * ct};
            for (int ax = 0; ax < 3; ++ax) {
                double v = pos[ax], q = mom[ax];
                if (p->fp32) { v = (double)(float)v; q = (double)(float)q; }
                st[ax * n + g] = v;
                st[(3 + ax) * n + g] = q;
            }
        }
        g0 += counts[r];
    }
    free(counts);
    return ORC_OK;
}

/*
 * Hot-spot initial state (the 3D thermal-box workload; the paper's runs use
 * two temperatures, this profile is the library's reading of a "Gaussian hot
 * spot"): T(r) = T0 + dT exp(-|r - centre|^2 / (2 w^2)) about the box centre,
 * density proportional to T(r)^3.  Particle g places itself by rejection:
 * try k = 0, 1, ... draws the block (STEP_INIT, g_lo, g_hi, 2 + k) with words
 * 0..2 a uniform position in the box and word 3 the acceptance variate,
 * accepted iff u < (T(r)/(T0 + dT))^3; after 64 rejected tries the 64th
 * position is kept.  Momentum as in orc_init_thermal at the local T(r):
 * E = -T ln(u1 u2 u3) with u1 = word 3 of block (STEP_INIT, g_lo, g_hi, 0) and
 * u2, u3 = words 0, 1 of block (..., 1); direction from words 2, 3 of (..., 1).
 */
int orc_init_hotspot(const orc_params *p, int64_t n, double T0, double dT, double width, double *st)
{
    if (check_params(p) != ORC_OK || !(T0 > 0.0) || !(dT >= 0.0) || !(width > 0.0)) return ORC_ERR_INVALID;
    const double Tmax = T0 + dT;
    const double c[3] = {0.5 * p->L[0], 0.5 * p->L[1], 0.5 * p->L[2]};
    for (int64_t g = 0; g < n; ++g) {
        uint32_t glo = (uint32_t)g, ghi = (uint32_t)((uint64_t)g >> 32);
        double pos[3] = {0.0, 0.0, 0.0};
        double T = T0;
        for (uint32_t k = 0; k < 64; ++k) {
            uint32_t t[4];
            philox(STEP_INIT, glo, ghi, 2u + k, p->key, t);
            double r2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                pos[a] = open01(t[a]) * p->L[a];
                double d = pos[a] - c[a];
                r2 += d * d;
            }
            T = T0 + dT * exp(-r2 / (2.0 * width * width));
            double ratio = T / Tmax;
            if (open01(t[3]) < ratio * ratio * ratio) break;
        }
        uint32_t a[4], b[4];
        philox(STEP_INIT, glo, ghi, 0u, p->key, a);
        philox(STEP_INIT, glo, ghi, 1u, p->key, b);
        double E = sample_pmag(p, T, glo, ghi, -T * log(open01(a[3]) * open01(b[0]) * open01(b[1])));
        double ct = 2.0 * open01(b[2]) - 1.0;
        double stt = sqrt((1.0 - ct) * (1.0 + ct));
        double phi = 2.0 * M_PI * open01(b[3]);
        double mom[3] = {E * stt * cos(phi), E * stt * sin(phi), E * ct};
        for (int ax = 0; ax < 3; ++ax) {
            double v = pos[ax], q = mom[ax];
            if (p->fp32) { v = (double)(float)v; q = (double)(float)q; }
            st[ax * n + g] = v;
            st[(3 + ax) * n + g] = q;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* A1-A3: free streaming (Eq. 2), wall reflection, cell key                  */
/* ------------------------------------------------------------------------ */

/* Cell key of one position, FP64: ix = clamp(floor(x / dx), 0, nx - 1). */
static uint32_t key_d(const orc_params *p, double x, double y, double z)
{
    double q[3] = {x, y, z};
    int64_t idx[3];
    for (int a = 0; a < 3; ++a) {
        double c = floor(q[a] / cell_len(p, a));
        int64_t ic;
        if (c < 0.0) ic = 0;
        else if (c >= (double)p->n[a]) ic = p->n[a] - 1;
        else ic = (int64_t)c;
        idx[a] = ic;
    }
    return (uint32_t)(idx[0] + (int64_t)p->n[0] * (idx[1] + (int64_t)p->n[1] * idx[2]));
}

/* Same in single precision: positions and dx are floats, division is IEEE. */
static uint32_t key_f(const orc_params *p, float x, float y, float z)
{
    float q[3] = {x, y, z};
    int64_t idx[3];
    for (int a = 0; a < 3; ++a) {
        float d = (float)cell_len(p, a);
        float c = floorf(q[a] / d);
        int64_t ic;
        if (c < 0.0f) ic = 0;
        else if (c >= (float)p->n[a]) ic = p->n[a] - 1;
        else ic = (int64_t)c;
        idx[a] = ic;
    }
    return (uint32_t)(idx[0] + (int64_t)p->n[0] * (idx[1] + (int64_t)p->n[1] * idx[2]));
}

/* Cell keys of a state without moving it. */
int orc_keys(const orc_params *p, int64_t n, const double *st, uint32_t *keys)
{
    if (check_params(p) != ORC_OK) return ORC_ERR_INVALID;
    for (int64_t k = 0; k < n; ++k) {
        if (p->fp32)
            keys[k] = key_f(p, (float)st[k], (float)st[n + k], (float)st[2 * n + k]);
        else
            keys[k] = key_d(p, st[k], st[n + k], st[2 * n + k]);
    }
    return ORC_OK;
}

/*
 * Stream one particle for dt and reflect it at the walls, FP64.
 * x <- x + (p_x / E) dt (Eq. 2 with c = 1, E = sqrt(|p|^2 + m^2));
 * a particle beyond a wall is mirrored back and its momentum component flips
 * (elastic reflection, Sec. 2).  A particle exactly on a wall stays there.
 * Returns the number of reflections.
 */
static int stream_d(const orc_params *p, double *pos, double *mom)
{
    double E = sqrt(((mom[0] * mom[0] + mom[1] * mom[1]) + mom[2] * mom[2]) + p->mass * p->mass);
    int nref = 0;
    for (int a = 0; a < 3; ++a) {
        double v = (E > 0.0) ? (mom[a] / E) : 0.0;
        double x = pos[a] + v * p->dt;
        if (x < 0.0) {
            x = -x;
            mom[a] = -mom[a];
            ++nref;
        } else if (x > p->L[a]) {
            x = (p->L[a] + p->L[a]) - x;
            mom[a] = -mom[a];
            ++nref;
        }
        pos[a] = x;
    }
    return nref;
}

/* Same in single precision (dt, L and m^2 rounded to float once). */
static int stream_f(const orc_params *p, float *pos, float *mom)
{
    float E = sqrtf(((mom[0] * mom[0] + mom[1] * mom[1]) + mom[2] * mom[2]) + (float)(p->mass * p->mass));
    float dt = (float)p->dt;
    int nref = 0;
    for (int a = 0; a < 3; ++a) {
        float L = (float)p->L[a];
        float v = (E > 0.0f) ? (mom[a] / E) : 0.0f;
        float x = pos[a] + v * dt;
        if (x < 0.0f) {
            x = -x;
            mom[a] = -mom[a];
            ++nref;
        } else if (x > L) {
            x = (L + L) - x;
            mom[a] = -mom[a];
            ++nref;
        }
        pos[a] = x;
    }
    return nref;
}

/* ------------------------------------------------------------------------ */
/* A4: stable counting sort by cell key                                      */
/* ------------------------------------------------------------------------ */

/*
 * Stable counting sort of the state by key: counts per cell, exclusive prefix
 * sum into cell_start, then every particle in array order goes to the next
 * free slot of its cell.  perm[k] = old index of the particle now at k.
 */
static int sort_by_key(const orc_params *p, int64_t n, double *st, const uint32_t *keys,
                       int64_t *perm_out, int64_t *cell_start_out)
{
    int64_t nc = orc_ncells(p);
    int64_t *start = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!start || !fill || !perm || !tmp) {
        free(start); free(fill); free(perm); free(tmp);
        return ORC_ERR_OOM;
    }
    for (int64_t k = 0; k < n; ++k) start[keys[k] + 1] += 1;
    for (int64_t c = 0; c < nc; ++c) start[c + 1] += start[c];
    for (int64_t c = 0; c < nc; ++c) fill[c] = start[c];
    for (int64_t k = 0; k < n; ++k) perm[fill[keys[k]]++] = k;
    for (int comp = 0; comp < 6; ++comp) {
        double *col = st + (int64_t)comp * n;
        for (int64_t k = 0; k < n; ++k) tmp[k] = col[perm[k]];
        memcpy(col, tmp, sizeof(double) * (size_t)n);
    }
    if (perm_out) memcpy(perm_out, perm, sizeof(int64_t) * (size_t)n);
    if (cell_start_out) memcpy(cell_start_out, start, sizeof(int64_t) * (size_t)(nc + 1));
    free(start); free(fill); free(perm); free(tmp);
    return ORC_OK;
}

/* Sort a state by cell key (used after sampling or loading a state). */
int orc_sort(const orc_params *p, int64_t n, double *st, uint32_t *keys_out, int64_t *perm_out,
             int64_t *cell_start_out)
{
    if (check_params(p) != ORC_OK) return ORC_ERR_INVALID;
    uint32_t *keys = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    if (!keys) return ORC_ERR_OOM;
    orc_keys(p, n, st, keys);
    int rc = sort_by_key(p, n, st, keys, perm_out, cell_start_out);
    if (keys_out) memcpy(keys_out, keys, sizeof(uint32_t) * (size_t)n);
    free(keys);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* A5: pair test P22 = C v_rel against a uniform u_ij (Eq. 3)                */
/* ------------------------------------------------------------------------ */

/*
 * The 32-bit word r_ij behind u_ij = r_ij 2^-32 of pair (i, j), i < j, of a
 * cell, assembled from three independent Philox streams (the paper only says
 * "Monte-Carlo"; this layout is the library's reading):
 *   bits 31..24: byte (j mod 16) of the block (step, cell, i, j / 16),
 *   bits 23..16: byte (j mod 16) of the block (step, cell, i, TAG_MID | j / 16),
 *   bits 15..0:  the top 16 bits of word 0 of the block (step, cell, i, TAG_FINE | j),
 * bytes numbered little-endian across the four output words.  The three parts
 * are independent uniforms, so r_ij is a uniform 32-bit word.
 */
uint32_t orc_pair_word(const uint32_t key[2], uint32_t step, uint32_t cell, uint32_t i, uint32_t j)
{
    uint32_t a[4], m[4], b[4];
    philox(step, cell, i, j >> 4, key, a);
    philox(step, cell, i, TAG_MID | (j >> 4), key, m);
    uint32_t top = (a[(j >> 2) & 3u] >> (8u * (j & 3u))) & 0xFFu;
    uint32_t mid = (m[(j >> 2) & 3u] >> (8u * (j & 3u))) & 0xFFu;
    philox(step, cell, i, TAG_FINE | j, key, b);
    return (top << 24) | (mid << 16) | (b[0] >> 16);
}

/* Unit direction p/E of a massless particle (zero vector if p = 0). */
static void unit_d(const double *m, double *u)
{
    double E = sqrt((m[0] * m[0] + m[1] * m[1]) + m[2] * m[2]);
    for (int a = 0; a < 3; ++a) u[a] = (E > 0.0) ? (m[a] / E) : 0.0;
}

static void unit_f(const float *m, float *u)
{
    float E = sqrtf((m[0] * m[0] + m[1] * m[1]) + m[2] * m[2]);
    for (int a = 0; a < 3; ++a) u[a] = (E > 0.0f) ? (m[a] / E) : 0.0f;
}

/*
 * v_rel = s / (2 E_i E_j) for massless particles (Sec. 2) equals
 * 1 - n_i . n_j = |n_i - n_j|^2 / 2; the difference form is used.
 */
static double vrel_d(const double *ui, const double *uj)
{
    double d0 = ui[0] - uj[0], d1 = ui[1] - uj[1], d2 = ui[2] - uj[2];
    return 0.5 * ((d0 * d0 + d1 * d1) + d2 * d2);
}

static float vrel_f(const float *ui, const float *uj)
{
    float d0 = ui[0] - uj[0], d1 = ui[1] - uj[1], d2 = ui[2] - uj[2];
    return 0.5f * ((d0 * d0 + d1 * d1) + d2 * d2);
}

/*
 * v_rel of massive particles (mass m): s / (2 E_i E_j) generalises to the
 * Moller velocity sqrt((p_i.p_j)^2 - m^4) / (E_i E_j) with the four-vector
 * product p_i.p_j = E_i E_j - p_i.p_j (3-vectors), written
 * sqrt((F - m^2)(F + m^2)) / (E_i E_j); 0 where rounding makes F < m^2.
 */
static double vrel_massive_d(double m2, const double *mi, const double *mj)
{
    double Ei = sqrt(((mi[0] * mi[0] + mi[1] * mi[1]) + mi[2] * mi[2]) + m2);
    double Ej = sqrt(((mj[0] * mj[0] + mj[1] * mj[1]) + mj[2] * mj[2]) + m2);
    double F = Ei * Ej - ((mi[0] * mj[0] + mi[1] * mj[1]) + mi[2] * mj[2]);
    double a = F - m2;
    if (!(a > 0.0)) return 0.0;
    return sqrt(a * (F + m2)) / (Ei * Ej);
}

static float vrel_massive_f(float m2, const float *mi, const float *mj)
{
    float Ei = sqrtf(((mi[0] * mi[0] + mi[1] * mi[1]) + mi[2] * mi[2]) + m2);
    float Ej = sqrtf(((mj[0] * mj[0] + mj[1] * mj[1]) + mj[2] * mj[2]) + m2);
    float F = Ei * Ej - ((mi[0] * mj[0] + mi[1] * mj[1]) + mi[2] * mj[2]);
    float a = F - m2;
    if (!(a > 0.0f)) return 0.0f;
    return sqrtf(a * (F + m2)) / (Ei * Ej);
}

/* P22 = C v_rel of a pair in the state's precision (massless: the unit-vector
   form; massive: the Moller velocity). */
static double p22_d(const orc_params *p, double C, const double *mi, const double *mj)
{
    if (p->mass > 0.0) return C * vrel_massive_d(p->mass * p->mass, mi, mj);
    double ui[3], uj[3];
    unit_d(mi, ui);
    unit_d(mj, uj);
    return C * vrel_d(ui, uj);
}

static float p22_f(const orc_params *p, double C, const double *mi, const double *mj)
{
    float fi[3] = {(float)mi[0], (float)mi[1], (float)mi[2]};
    float fj[3] = {(float)mj[0], (float)mj[1], (float)mj[2]};
    if (p->mass > 0.0) return (float)C * vrel_massive_f((float)(p->mass * p->mass), fi, fj);
    float ui[3], uj[3];
    unit_f(fi, ui);
    unit_f(fj, uj);
    return (float)C * vrel_f(ui, uj);
}

/* Accept pair (i, j) iff u_ij < P22, evaluated in the state's precision. */
static int accept_pair(const orc_params *p, double C, uint32_t step, uint32_t cell, uint32_t i,
                       uint32_t j, const double *mi, const double *mj)
{
    uint32_t r = orc_pair_word(p->key, step, cell, i, j);
    if (p->fp32) {
        float u = (float)r * 0x1p-32f;
        return u < p22_f(p, C, mi, mj);
    } else {
        double u = (double)r * 0x1p-32;
        return u < p22_d(p, C, mi, mj);
    }
}

/* ------------------------------------------------------------------------ */
/* A5, skip-ahead mode: Bernoulli candidates with geometric gaps, thinning   */
/* ------------------------------------------------------------------------ */

/*
 * The paper tests every pair with its own uniform (Eq. 3).  The skip-ahead
 * mode draws the same accepted-pair distribution with work proportional to
 * the number of candidates: along row i (columns j = i+1 .. n-1 in order) a
 * pair is a candidate with probability P_max >= max P22 independently of the
 * others, so the gaps between candidates are geometric; a candidate is then
 * kept with probability P22 / P_max (thinning).  Each pair ends up accepted
 * with probability P22, independently, as in the all-pairs test; only the
 * realisation differs.
 *
 * Reading (exact, integer-only where it decides an index):
 *  - P_max: P_fix = floor(2.0001 C 2^64) (at least 1) as a 0.64 fixed-point
 *    fraction; q = 2^64 - P_fix is 1 - P_max; Q[b] = q^(2^b) by repeated
 *    truncated fixed-point squaring, b = 0 .. 32;
 *  - the k-th draw of row i is the Philox block (step, cell, i, TAG_SKIP | k):
 *    U = word0 2^32 + word1 (64-bit uniform), w = word2 (thinning);
 *  - gap: with pos the last candidate (i at the start) and M = n - 1 - pos
 *    columns left, G = the largest integer < 2^(bt+1) whose fixed-point power
 *    q^G, built greedily from bit bt = ceil(log2 M) down to bit 0, is still
 *    >= U: P(G >= k) = q^k up to rounding (inverse-CDF of the geometric
 *    distribution).  G >= M ends the row; otherwise j = pos + 1 + G;
 *  - thinning: accept iff (unit(w) * P_max) < P22 in the state's precision,
 *    with P_max = P_fix 2^-64 rounded to that precision and unit(w) = w 2^-32.
 */
static uint64_t mulhi64(uint64_t a, uint64_t b)
{
    return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
}

int orc_skip_table(double C, uint64_t *p_fix, uint64_t Q[33])
{
    double x = 2.0001 * C;
    if (!(x > 0.0) || !(x < 1.0)) return ORC_ERR_INVALID;
    uint64_t P = (uint64_t)ldexp(x, 64);
    if (P == 0) P = 1;
    *p_fix = P;
    Q[0] = (uint64_t)0 - P;
    for (int b = 1; b <= 32; ++b) Q[b] = mulhi64(Q[b - 1], Q[b - 1]);
    return ORC_OK;
}

uint64_t orc_skip_gap(const uint64_t Q[33], uint64_t U, uint64_t M)
{
    int bt = 0;
    while (bt < 32 && ((uint64_t)1 << bt) < M) ++bt;
    uint64_t G = 0, Qc = ~(uint64_t)0;
    for (int b = bt; b >= 0; --b) {
        uint64_t t = mulhi64(Qc, Q[b]);
        if (t >= U) {
            Qc = t;
            G += (uint64_t)1 << b;
        }
    }
    return G;
}

/* Thinning of candidate (i, j) with word w: accept iff unit(w) P_max < P22. */
static int thin_accept(const orc_params *p, double C, uint64_t P_fix, uint32_t w, const double *mi,
                       const double *mj)
{
    double Pm = (double)P_fix * 0x1p-64;
    if (p->fp32) {
        float u = ((float)w * 0x1p-32f) * (float)Pm;
        return u < p22_f(p, C, mi, mj);
    } else {
        double u = ((double)w * 0x1p-32) * Pm;
        return u < p22_d(p, C, mi, mj);
    }
}

/*
 * Candidates of row i of a cell of nc particles (momenta px, py, pz in sorted
 * order), in increasing j; accepted columns go to out_j (at most cap written).
 * Returns the number accepted; *n_cand receives the number of candidates.
 */
static int64_t skip_row(const orc_params *p, double C, uint64_t P_fix, const uint64_t Q[33], uint32_t step,
                        uint32_t cell, int64_t nc, int64_t i, const double *px, const double *py,
                        const double *pz, uint32_t *out_j, int64_t cap, int64_t *n_cand)
{
    int64_t pos = i, count = 0, cand = 0;
    double mi[3] = {px[i], py[i], pz[i]};
    for (uint32_t k = 0;; ++k) {
        uint64_t M = (uint64_t)(nc - 1 - pos);
        if (M == 0) break;
        uint32_t w[4];
        philox(step, cell, (uint32_t)i, TAG_SKIP | k, p->key, w);
        uint64_t U = ((uint64_t)w[0] << 32) | w[1];
        uint64_t G = orc_skip_gap(Q, U, M);
        if (G >= M) break;
        int64_t j = pos + 1 + (int64_t)G;
        double mj[3] = {px[j], py[j], pz[j]};
        ++cand;
        if (thin_accept(p, C, P_fix, w[2], mi, mj)) {
            if (out_j && count < cap) out_j[count] = (uint32_t)j;
            ++count;
        }
        pos = j;
    }
    if (n_cand) *n_cand = cand;
    return count;
}

/* ------------------------------------------------------------------------ */
/* A7: kinematics — boost to the CM frame, isotropic direction, boost back   */
/* ------------------------------------------------------------------------ */

/*
 * New momenta of an executed pair (Sec. 2).  With P = p_i + p_j,
 * E_t = E_i + E_j, beta = P / E_t, gamma = E_t / sqrt(s): in the CM frame
 * both particles carry E* = sqrt(s)/2 and momenta +-p*, |p*| =
 * sqrt(E*^2 - m^2) (massless: s = 2 E_i E_j v_rel and |p*| = E*).  Boosting
 * back: p' = p* + beta (gamma^2/(gamma+1) (beta . p*) + gamma E*).
 * The direction of p* comes from the Philox block (step, cell, i,
 * TAG_ANGLE | j), u1 = word0 2^-32, u2 = word1 2^-32, phi = 2 pi u2:
 *  - isotropic (mu = 0, the paper's case): cos t = 2 u1 - 1 about the z axis;
 *  - screened forward peak (mu > 0, no counterpart in the paper; the
 *    pQCD-like dsigma/dt ~ 1/(t - mu^2)^2 with t = -2 |p*|^2 (1 - cos t)):
 *    x = 1 - cos t by inverting its CDF in closed form, with a = 2 |p*|^2,
 *    A = 1/mu^2, B = 1/(2a + mu^2): x = (1/(A - u1 (A - B)) - mu^2) / a, the
 *    angle measured from the incoming CM direction of particle i (its
 *    momentum boosted by -beta: p_i + beta (gamma^2/(gamma+1) (beta . p_i)
 *    - gamma E_i)), phi about it in the basis e1 = unit(h x e),
 *    e2 = e x e1 with h = x^ if |e_x| < 0.9, else y^.
 * The total cross section (and P22) is the same in both cases.  Returns 0
 * if s <= 4 m^2 (nothing happens).
 */
static int kin_general(const uint32_t key[2], double mass, double mu, uint32_t step, uint32_t cell, uint32_t i,
                       uint32_t j, double *mi, double *mj)
{
    const double m2 = mass * mass;
    double Ei = sqrt(((mi[0] * mi[0] + mi[1] * mi[1]) + mi[2] * mi[2]) + m2);
    double Ej = sqrt(((mj[0] * mj[0] + mj[1] * mj[1]) + mj[2] * mj[2]) + m2);
    double s;
    if (mass > 0.0) {
        double F = Ei * Ej - ((mi[0] * mj[0] + mi[1] * mj[1]) + mi[2] * mj[2]);
        s = 2.0 * m2 + 2.0 * F;
        if (!(s > 4.0 * m2)) return 0;
    } else {
        double ui[3], uj[3];
        unit_d(mi, ui);
        unit_d(mj, uj);
        s = ((2.0 * Ei) * Ej) * vrel_d(ui, uj);
        if (!(s > 0.0)) return 0;
    }
    double rs = sqrt(s);
    double Es = 0.5 * rs;
    double ps_mag = mass > 0.0 ? sqrt((Es - mass) * (Es + mass)) : Es;
    double Et = Ei + Ej;
    double beta[3] = {(mi[0] + mj[0]) / Et, (mi[1] + mj[1]) / Et, (mi[2] + mj[2]) / Et};
    double gamma = Et / rs;
    double a = (gamma * gamma) / (gamma + 1.0);
    uint32_t w[4];
    philox(step, cell, i, TAG_ANGLE | j, key, w);
    double u1 = (double)w[0] * 0x1p-32, u2 = (double)w[1] * 0x1p-32;
    double phi = 2.0 * M_PI * u2;
    double ps[3];
    if (!(mu > 0.0)) {
        double ct = 2.0 * u1 - 1.0;
        double stt = sqrt((1.0 - ct) * (1.0 + ct));
        ps[0] = ps_mag * (stt * cos(phi));
        ps[1] = ps_mag * (stt * sin(phi));
        ps[2] = ps_mag * ct;
    } else {
        /* incoming CM direction of particle i */
        double bpi = (beta[0] * mi[0] + beta[1] * mi[1]) + beta[2] * mi[2];
        double fi_in = a * bpi - gamma * Ei;
        double e[3] = {mi[0] + beta[0] * fi_in, mi[1] + beta[1] * fi_in, mi[2] + beta[2] * fi_in};
        double en = sqrt((e[0] * e[0] + e[1] * e[1]) + e[2] * e[2]);
        for (int ax = 0; ax < 3; ++ax) e[ax] = e[ax] / en;
        double h[3] = {0.0, 0.0, 0.0};
        if (fabs(e[0]) < 0.9) h[0] = 1.0; else h[1] = 1.0;
        double e1[3] = {h[1] * e[2] - h[2] * e[1], h[2] * e[0] - h[0] * e[2], h[0] * e[1] - h[1] * e[0]};
        double n1 = sqrt((e1[0] * e1[0] + e1[1] * e1[1]) + e1[2] * e1[2]);
        for (int ax = 0; ax < 3; ++ax) e1[ax] = e1[ax] / n1;
        double e2[3] = {e[1] * e1[2] - e[2] * e1[1], e[2] * e1[0] - e[0] * e1[2], e[0] * e1[1] - e[1] * e1[0]};
        double aa = 2.0 * (ps_mag * ps_mag);
        double mu2 = mu * mu;
        double A = 1.0 / mu2, B = 1.0 / (2.0 * aa + mu2);
        double x = (1.0 / (A - u1 * (A - B)) - mu2) / aa;
        if (x < 0.0) x = 0.0;
        if (x > 2.0) x = 2.0;
        double ct = 1.0 - x;
        double stt = sqrt(x * (2.0 - x));
        double cp = cos(phi), sp = sin(phi);
        for (int ax = 0; ax < 3; ++ax)
            ps[ax] = ps_mag * (ct * e[ax] + stt * (cp * e1[ax] + sp * e2[ax]));
    }
    double bp = (beta[0] * ps[0] + beta[1] * ps[1]) + beta[2] * ps[2];
    double fi = a * bp + gamma * Es;
    double fj = -a * bp + gamma * Es;
    for (int ax = 0; ax < 3; ++ax) {
        mi[ax] = ps[ax] + beta[ax] * fi;
        mj[ax] = -ps[ax] + beta[ax] * fj;
    }
    return 1;
}

/* Massless particles, isotropic direction (the paper's case). */
int orc_kinematics(const uint32_t key[2], uint32_t step, uint32_t cell, uint32_t i, uint32_t j, double *mi,
                   double *mj)
{
    return kin_general(key, 0.0, 0.0, step, cell, i, j, mi, mj);
}

/* Any mass and angular distribution (mass, mu as in orc_params). */
int orc_kinematics_ex(const uint32_t key[2], double mass, double mu, uint32_t step, uint32_t cell, uint32_t i,
                      uint32_t j, double *mi, double *mj)
{
    return kin_general(key, mass, mu, step, cell, i, j, mi, mj);
}

/* ------------------------------------------------------------------------ */
/* A5-A7 for one cell                                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint32_t *acc; /* accepted pairs (i, j) in lexicographic order */
    int64_t n_acc, cap;
    uint8_t *exe;  /* executed flag per accepted pair */
    int64_t n_exe;
    int64_t n_cand; /* skip-ahead candidates */
} cell_result;

static int push_pair(cell_result *cr, uint32_t i, uint32_t j)
{
    if (cr->n_acc == cr->cap) {
        int64_t nc = cr->cap ? 2 * cr->cap : 64;
        uint32_t *na = (uint32_t *)realloc(cr->acc, sizeof(uint32_t) * 2 * (size_t)nc);
        if (!na) return ORC_ERR_OOM;
        cr->acc = na;
        cr->cap = nc;
    }
    cr->acc[2 * cr->n_acc] = i;
    cr->acc[2 * cr->n_acc + 1] = j;
    cr->n_acc += 1;
    return ORC_OK;
}

/*
 * One cell of nc particles whose momenta sit at m[0..nc), m[nc..2nc),
 * m[2nc..3nc) (components px, py, pz), in sorted order:
 *  (1) test every pair i < j in lexicographic order and keep the accepted
 *      ones (A5) — or, in the skip-ahead mode, draw each row's candidates and
 *      thin them, which yields the accepted pairs in the same order;
 *  (2) walk the accepted pairs in that order and execute a pair iff neither
 *      particle has collided yet in this step (A6, greedy reading);
 *  (3) apply the kinematics to each executed pair (A7).
 */
static int do_cell(const orc_params *p, double C, uint32_t step, uint32_t cell, int64_t nc,
                   double *px, double *py, double *pz, cell_result *cr)
{
    memset(cr, 0, sizeof(*cr));
    if (nc < 2 || !(C > 0.0)) return ORC_OK;
    if (p->skip) {
        uint64_t P_fix, Q[33];
        if (orc_skip_table(C, &P_fix, Q) != ORC_OK) return ORC_ERR_INVALID;
        uint32_t *row = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)nc);
        if (!row) return ORC_ERR_OOM;
        for (int64_t i = 0; i + 1 < nc; ++i) {
            int64_t cand = 0;
            int64_t m = skip_row(p, C, P_fix, Q, step, cell, nc, i, px, py, pz, row, nc, &cand);
            cr->n_cand += cand;
            for (int64_t e = 0; e < m; ++e) {
                int rc = push_pair(cr, (uint32_t)i, row[e]);
                if (rc != ORC_OK) { free(row); return rc; }
            }
        }
        free(row);
    } else {
        for (int64_t i = 0; i < nc; ++i) {
            double mi[3] = {px[i], py[i], pz[i]};
            for (int64_t j = i + 1; j < nc; ++j) {
                double mj[3] = {px[j], py[j], pz[j]};
                if (accept_pair(p, C, step, cell, (uint32_t)i, (uint32_t)j, mi, mj)) {
                    int rc = push_pair(cr, (uint32_t)i, (uint32_t)j);
                    if (rc != ORC_OK) return rc;
                }
            }
        }
    }
    if (cr->n_acc == 0) return ORC_OK;
    cr->exe = (uint8_t *)calloc((size_t)cr->n_acc, 1);
    uint8_t *used = (uint8_t *)calloc((size_t)nc, 1);
    if (!cr->exe || !used) { free(used); return ORC_ERR_OOM; }
    for (int64_t e = 0; e < cr->n_acc; ++e) {
        uint32_t i = cr->acc[2 * e], j = cr->acc[2 * e + 1];
        if (used[i] || used[j]) continue;
        used[i] = 1;
        used[j] = 1;
        cr->exe[e] = 1;
        cr->n_exe += 1;
        double mi[3] = {px[i], py[i], pz[i]};
        double mj[3] = {px[j], py[j], pz[j]};
        kin_general(p->key, p->mass, p->mu, step, cell, i, j, mi, mj);
        if (p->fp32) {
            for (int a = 0; a < 3; ++a) { mi[a] = (double)(float)mi[a]; mj[a] = (double)(float)mj[a]; }
        }
        px[i] = mi[0]; py[i] = mi[1]; pz[i] = mi[2];
        px[j] = mj[0]; py[j] = mj[1]; pz[j] = mj[2];
    }
    free(used);
    return ORC_OK;
}

/*
 * Accepted pairs of one cell, for sampled comparisons at sizes where a whole
 * step is out of reach: momenta of the cell's nc particles in sorted order,
 * output (i, j) pairs in lexicographic order (at most cap are written; the
 * return value is the total count, or a negative error).
 */
int64_t orc_cell_accept(const orc_params *p, uint32_t step, uint32_t cell, int64_t nc,
                        const double *px, const double *py, const double *pz, uint32_t *out_ij,
                        int64_t cap)
{
    if (check_params(p) != ORC_OK) return ORC_ERR_INVALID;
    double C = orc_p22_scale(p);
    int64_t count = 0;
    if (!(C > 0.0)) return 0;
    if (p->skip) {
        uint64_t P_fix, Q[33];
        if (orc_skip_table(C, &P_fix, Q) != ORC_OK) return ORC_ERR_INVALID;
        uint32_t *row = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nc > 0 ? nc : 1));
        if (!row) return ORC_ERR_OOM;
        for (int64_t i = 0; i + 1 < nc; ++i) {
            int64_t m = skip_row(p, C, P_fix, Q, step, cell, nc, i, px, py, pz, row, nc, NULL);
            for (int64_t e = 0; e < m; ++e, ++count) {
                if (count < cap && out_ij) {
                    out_ij[2 * count] = (uint32_t)i;
                    out_ij[2 * count + 1] = row[e];
                }
            }
        }
        free(row);
        return count;
    }
    for (int64_t i = 0; i < nc; ++i) {
        double mi[3] = {px[i], py[i], pz[i]};
        for (int64_t j = i + 1; j < nc; ++j) {
            double mj[3] = {px[j], py[j], pz[j]};
            if (accept_pair(p, C, step, cell, (uint32_t)i, (uint32_t)j, mi, mj)) {
                if (count < cap && out_ij) {
                    out_ij[2 * count] = (uint32_t)i;
                    out_ij[2 * count + 1] = (uint32_t)j;
                }
                ++count;
            }
        }
    }
    return count;
}

/* Pair tests of one cell row i only (columns j in [j0, j1)), for sampling. */
int64_t orc_row_accept(const orc_params *p, uint32_t step, uint32_t cell, int64_t nc, int64_t i,
                       int64_t j0, int64_t j1, const double *px, const double *py, const double *pz,
                       uint32_t *out_j, int64_t cap)
{
    if (check_params(p) != ORC_OK) return ORC_ERR_INVALID;
    double C = orc_p22_scale(p);
    int64_t count = 0;
    if (!(C > 0.0) || i < 0 || i >= nc) return 0;
    if (j0 < i + 1) j0 = i + 1;
    if (j1 > nc) j1 = nc;
    if (p->skip) {
        /* the row's candidate process starts at column i + 1 whatever the
           window: draw the whole row, keep the columns in [j0, j1) */
        uint64_t P_fix, Q[33];
        if (orc_skip_table(C, &P_fix, Q) != ORC_OK) return ORC_ERR_INVALID;
        uint32_t *row = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)nc);
        if (!row) return ORC_ERR_OOM;
        int64_t m = skip_row(p, C, P_fix, Q, step, cell, nc, i, px, py, pz, row, nc, NULL);
        for (int64_t e = 0; e < m; ++e) {
            if (row[e] < (uint32_t)j0 || row[e] >= (uint32_t)j1) continue;
            if (count < cap && out_j) out_j[count] = row[e];
            ++count;
        }
        free(row);
        return count;
    }
    double mi[3] = {px[i], py[i], pz[i]};
    for (int64_t j = j0; j < j1; ++j) {
        double mj[3] = {px[j], py[j], pz[j]};
        if (accept_pair(p, C, step, cell, (uint32_t)i, (uint32_t)j, mi, mj)) {
            if (count < cap && out_j) out_j[count] = (uint32_t)j;
            ++count;
        }
    }
    return count;
}

/* ------------------------------------------------------------------------ */
/* Adaptive time step                                                        */
/* ------------------------------------------------------------------------ */

/*
 * The paper leaves a variable dt to future work (Sec. 6).  Reading: with
 * kappa > 0 each step's dt is taken at its start from the sorted state so that
 * a particle of the most populated cell (n_max particles) expects about kappa
 * collisions in the step: (n_max - 1) C <v_rel> = kappa with <v_rel> = 1 for
 * an isotropic massless gas and C = sigma dt / (N_test V_cell) (Eq. 3), i.e.
 *   dt = ((kappa N_test) V_cell) / (sigma (n_max - 1)),
 * capped by the given dt (below every cell edge, Sec. 5).  Without
 * collisions (sigma = 0, or n_max < 2) the cap is used.  kappa <= 1/2 keeps
 * 2 C <= 1.
 */
double orc_adaptive_dt(const orc_params *p, int64_t n_max)
{
    if (!(p->kappa > 0.0) || !(p->sigma > 0.0) || n_max < 2) return p->dt;
    double dt = ((p->kappa * p->n_test) * cell_volume(p)) / (p->sigma * (double)(n_max - 1));
    return dt < p->dt ? dt : p->dt;
}

/* Largest cell population of a state (keys in the state's precision). */
static int64_t max_cell_count(const orc_params *p, int64_t n, const double *st)
{
    int64_t ncell = orc_ncells(p);
    int64_t *cnt = (int64_t *)calloc((size_t)ncell, sizeof(int64_t));
    if (!cnt) return -1;
    for (int64_t k = 0; k < n; ++k) {
        uint32_t key = p->fp32 ? key_f(p, (float)st[k], (float)st[n + k], (float)st[2 * n + k])
                               : key_d(p, st[k], st[n + k], st[2 * n + k]);
        cnt[key] += 1;
    }
    int64_t m = 0;
    for (int64_t c = 0; c < ncell; ++c) m = cnt[c] > m ? cnt[c] : m;
    free(cnt);
    return m;
}

/* ------------------------------------------------------------------------ */
/* One full time step                                                        */
/* ------------------------------------------------------------------------ */

/*
 * Advance a state (sorted by cell, layout as in orc_init_thermal) by one time
 * step with random-stream step index `step`: A1-A3 stream/reflect/key for
 * every particle, A4 stable sort, A5-A7 collisions cell by cell.  Positions
 * are not changed by collisions.  The optional trace receives the details.
 */
int orc_step(const orc_params *p_in, uint32_t step, int64_t n, double *st, orc_trace *tr)
{
    if (check_params(p_in) != ORC_OK) return ORC_ERR_INVALID;
    /* the step's dt: the given one, or the adaptive choice from the state */
    orc_params q = *p_in;
    if (q.kappa > 0.0) {
        int64_t nmax = max_cell_count(p_in, n, st);
        if (nmax < 0) return ORC_ERR_OOM;
        q.dt = orc_adaptive_dt(p_in, nmax);
    }
    const orc_params *p = &q;
    if (tr) tr->dt = q.dt;
    int64_t ncell = orc_ncells(p);
    uint32_t *keys = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *cs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncell + 1));
    if (!keys || !cs) { free(keys); free(cs); return ORC_ERR_OOM; }
    int64_t nref = 0;

#pragma omp parallel for reduction(+ : nref) schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        if (p->fp32) {
            float pos[3] = {(float)st[k], (float)st[n + k], (float)st[2 * n + k]};
            float mom[3] = {(float)st[3 * n + k], (float)st[4 * n + k], (float)st[5 * n + k]};
            nref += stream_f(p, pos, mom);
            for (int a = 0; a < 3; ++a) {
                st[a * n + k] = pos[a];
                st[(3 + a) * n + k] = mom[a];
            }
            keys[k] = key_f(p, pos[0], pos[1], pos[2]);
        } else {
            double pos[3] = {st[k], st[n + k], st[2 * n + k]};
            double mom[3] = {st[3 * n + k], st[4 * n + k], st[5 * n + k]};
            nref += stream_d(p, pos, mom);
            for (int a = 0; a < 3; ++a) {
                st[a * n + k] = pos[a];
                st[(3 + a) * n + k] = mom[a];
            }
            keys[k] = key_d(p, pos[0], pos[1], pos[2]);
        }
    }
    if (tr && tr->keys) memcpy(tr->keys, keys, sizeof(uint32_t) * (size_t)n);

    int rc = sort_by_key(p, n, st, keys, tr ? tr->perm : NULL, cs);
    free(keys);
    if (rc != ORC_OK) { free(cs); return rc; }
    if (tr && tr->cell_start) memcpy(tr->cell_start, cs, sizeof(int64_t) * (size_t)(ncell + 1));

    double C = orc_p22_scale(p);
    cell_result *res = (cell_result *)calloc((size_t)ncell, sizeof(cell_result));
    if (!res) { free(cs); return ORC_ERR_OOM; }
    int err = ORC_OK;
    double *px = st + 3 * n, *py = st + 4 * n, *pz = st + 5 * n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < ncell; ++c) {
        int64_t b = cs[c], nc = cs[c + 1] - cs[c];
        int r = do_cell(p, C, step, (uint32_t)c, nc, px + b, py + b, pz + b, &res[c]);
        if (r != ORC_OK) {
#pragma omp critical
            err = r;
        }
    }
    if (tr) {
        tr->n_acc = 0;
        tr->n_exe = 0;
        tr->n_reflections = nref;
        tr->n_pairs_tested = 0;
        tr->n_candidates = 0;
    }
    for (int64_t c = 0; c < ncell; ++c) {
        cell_result *cr = &res[c];
        if (tr) {
            int64_t nc = cs[c + 1] - cs[c];
            tr->n_pairs_tested += (C > 0.0) ? nc * (nc - 1) / 2 : 0;
            tr->n_candidates += cr->n_cand;
            for (int64_t e = 0; e < cr->n_acc; ++e) {
                if (tr->acc && tr->n_acc < tr->acc_cap) {
                    tr->acc[3 * tr->n_acc] = (uint32_t)c;
                    tr->acc[3 * tr->n_acc + 1] = cr->acc[2 * e];
                    tr->acc[3 * tr->n_acc + 2] = cr->acc[2 * e + 1];
                }
                tr->n_acc += 1;
                if (cr->exe && cr->exe[e]) {
                    if (tr->exe && tr->n_exe < tr->exe_cap) {
                        tr->exe[3 * tr->n_exe] = (uint32_t)c;
                        tr->exe[3 * tr->n_exe + 1] = cr->acc[2 * e];
                        tr->exe[3 * tr->n_exe + 2] = cr->acc[2 * e + 1];
                    }
                    tr->n_exe += 1;
                }
            }
        }
        free(cr->acc);
        free(cr->exe);
    }
    free(res);
    free(cs);
    return err;
}

/* ------------------------------------------------------------------------ */
/* A8: observables                                                           */
/* ------------------------------------------------------------------------ */

/*
 * Per-cell energy density T^00 = sum E / (N_test V_cell), momentum density
 * T^0x = sum p_x / (N_test V_cell) and particle count, summed in FP64 in
 * sorted order; cell_start as produced by orc_sort / orc_step.
 */
int orc_observables(const orc_params *p, int64_t n, const double *st, const int64_t *cell_start,
                    double *T00, double *T0x, int32_t *counts)
{
    if (check_params(p) != ORC_OK) return ORC_ERR_INVALID;
    int64_t ncell = orc_ncells(p);
    double norm = p->n_test * cell_volume(p);
    for (int64_t c = 0; c < ncell; ++c) {
        double e = 0.0, m = 0.0;
        for (int64_t k = cell_start[c]; k < cell_start[c + 1]; ++k) {
            double qx = st[3 * n + k], qy = st[4 * n + k], qz = st[5 * n + k];
            e += sqrt(((qx * qx + qy * qy) + qz * qz) + p->mass * p->mass);
            m += qx;
        }
        if (T00) T00[c] = e / norm;
        if (T0x) T0x[c] = m / norm;
        if (counts) counts[c] = (int32_t)(cell_start[c + 1] - cell_start[c]);
    }
    return ORC_OK;
}

/* Total energy and momentum (FP64, particles of the given mass): out = {E, Px, Py, Pz}. */
void orc_totals(int64_t n, const double *st, double mass, double out[4])
{
    double e = 0.0, x = 0.0, y = 0.0, z = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        double qx = st[3 * n + k], qy = st[4 * n + k], qz = st[5 * n + k];
        e += sqrt(((qx * qx + qy * qy) + qz * qz) + mass * mass);
        x += qx;
        y += qy;
        z += qz;
    }
    out[0] = e; out[1] = x; out[2] = y; out[3] = z;
}

/* Number of OpenMP threads the oracle will use. */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
